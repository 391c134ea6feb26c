// fft.cu -- shared-memory FFTs for the Toeplitz (Gram) operator, its kernel
// spectrum, and the row passes of the CG iteration that fuse into them.
//
// T x = H^H H x is a 2-D linear convolution of x with conj(G) (Appendix B).
// Embedded in an M x M circulant (M >= 2N-1; the "circular convolution" of
// section 3.4 holds only after this zero padding) it becomes
//     T x = crop_N( IFFT2( Chat .* FFT2( pad_M(x) ) ) ),
// with Chat = FFT2(c) / M^2 real because c[-y][-x] = conj c[y][x] (the point
// symmetry of G).  The apply runs in three passes over an N x M buffer X:
//   rows:    N row FFTs of the zero-padded rows (N inputs, M outputs),
//   columns: per column FFT (N nonzero inputs) -> * Chat -> IFFT, rows < N,
//   rows:    N row IFFTs, columns < N kept.
// Inside the CG iteration the first row pass also forms the new direction
// d = -g + beta d_old and the first line-search sums, and the last row pass
// forms q2 = Re<d, T d> and the first line-search step (cg.cu holds the
// other CG kernels).
//
// FFTs are self-sorting Stockham transforms in shared memory.  For
// power-of-two M (the sizes the plan picks) the transform is compile-time:
// one radix-4 butterfly per thread per stage (plus one radix-2 stage for odd
// log2 M), values in registers between a read and a write phase.  Any other
// M = 2^a 3^b 5^c runs the runtime mixed-radix path with a ping-pong buffer.
#include <stdint.h>

#include "internal.cuh"
#include "phase.cuh"
#include "reduce.cuh"

namespace spirec {

bool make_fft_plan(int M, FftPlan* p)
{
    p->M = M;
    p->nstages = 0;
    int r = M;
    while (r > 1) {
        int rad;
        if (r % 4 == 0) rad = 4;
        else if (r % 2 == 0) rad = 2;
        else if (r % 3 == 0) rad = 3;
        else if (r % 5 == 0) rad = 5;
        else return false;
        if (p->nstages >= kMaxStages) return false;
        p->radix[p->nstages++] = rad;
        r /= rad;
    }
    return true;
}

namespace {

// ------------------------------------------------------------ small DFTs

// X[q] = sum_r v[r] w^(r q), w = exp(-+2 pi i / R).
template <int R, bool INV>
__device__ __forceinline__ void dft_small(float2* v)
{
    if (R == 2) {
        const float2 a = v[0], b = v[1];
        v[0] = make_float2(a.x + b.x, a.y + b.y);
        v[1] = make_float2(a.x - b.x, a.y - b.y);
    } else if (R == 4) {
        const float2 a = v[0], b = v[1], c = v[2], d = v[3];
        const float2 s0 = make_float2(a.x + c.x, a.y + c.y);
        const float2 s1 = make_float2(a.x - c.x, a.y - c.y);
        const float2 s2 = make_float2(b.x + d.x, b.y + d.y);
        const float2 s3 = make_float2(b.x - d.x, b.y - d.y);
        // forward: X1 = s1 - i s3, X3 = s1 + i s3; the inverse swaps them
        const float2 mis3 = INV ? make_float2(-s3.y, s3.x) : make_float2(s3.y, -s3.x);
        v[0] = make_float2(s0.x + s2.x, s0.y + s2.y);
        v[2] = make_float2(s0.x - s2.x, s0.y - s2.y);
        v[1] = make_float2(s1.x + mis3.x, s1.y + mis3.y);
        v[3] = make_float2(s1.x - mis3.x, s1.y - mis3.y);
    } else if (R == 3) {
        const float c1 = -0.5f;
        const float s1 = INV ? 0.86602540378443864676f : -0.86602540378443864676f;
        const float2 a = v[0], b = v[1], c = v[2];
        const float2 t = make_float2(b.x + c.x, b.y + c.y);
        const float2 u = make_float2(b.x - c.x, b.y - c.y);
        v[0] = make_float2(a.x + t.x, a.y + t.y);
        const float2 m = make_float2(a.x + c1 * t.x, a.y + c1 * t.y);
        v[1] = make_float2(m.x - s1 * u.y, m.y + s1 * u.x);
        v[2] = make_float2(m.x + s1 * u.y, m.y - s1 * u.x);
    } else {  // R == 5
        const float c1 = 0.30901699437494742410f, c2 = -0.80901699437494742410f;
        const float sg = INV ? 1.f : -1.f;
        const float s1 = sg * 0.95105651629515357212f, s2 = sg * 0.58778525229247312917f;
        const float2 a = v[0];
        const float2 b1 = make_float2(v[1].x + v[4].x, v[1].y + v[4].y);
        const float2 d1 = make_float2(v[1].x - v[4].x, v[1].y - v[4].y);
        const float2 b2 = make_float2(v[2].x + v[3].x, v[2].y + v[3].y);
        const float2 d2 = make_float2(v[2].x - v[3].x, v[2].y - v[3].y);
        v[0] = make_float2(a.x + b1.x + b2.x, a.y + b1.y + b2.y);
        const float2 m1 = make_float2(a.x + c1 * b1.x + c2 * b2.x, a.y + c1 * b1.y + c2 * b2.y);
        const float2 m2 = make_float2(a.x + c2 * b1.x + c1 * b2.x, a.y + c2 * b1.y + c1 * b2.y);
        const float2 e1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
        const float2 e2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
        v[1] = make_float2(m1.x - e1.y, m1.y + e1.x);
        v[4] = make_float2(m1.x + e1.y, m1.y - e1.x);
        v[2] = make_float2(m2.x - e2.y, m2.y + e2.x);
        v[3] = make_float2(m2.x + e2.y, m2.y - e2.x);
    }
}

__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e, bool inv)
{
    float2 w = __ldg(tw + e);
    if (inv) w.y = -w.y;
    return w;
}

// --------------------------------------------- runtime mixed-radix Stockham

template <int R, bool INV>
__device__ __forceinline__ void stage_rt(const float2* __restrict__ in, float2* __restrict__ out,
                                         int M, int Ns, int nseq, int ld,
                                         const float2* __restrict__ tw)
{
    const int nb = M / R;
    const int tstep = M / (Ns * R);
    for (int idx = threadIdx.x; idx < nseq * nb; idx += blockDim.x) {
        const int q = idx / nb, j = idx - q * nb;
        const float2* src = in + q * ld;
        float2* dst = out + q * ld;
        const int k = j % Ns;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twiddle(tw, k * r * tstep, INV));
        dft_small<R, INV>(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
    }
}

template <bool INV>
__device__ float2* fft_rt(float2* a, float2* b, const FftPlan& fp, int nseq, int ld,
                          const float2* __restrict__ tw)
{
    int Ns = 1;
    for (int s = 0; s < fp.nstages; ++s) {
        const int R = fp.radix[s];
        switch (R) {
        case 4: stage_rt<4, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        case 2: stage_rt<2, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        case 3: stage_rt<3, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        default: stage_rt<5, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// --------------------------------------------- compile-time power-of-two

__host__ __device__ constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// In-place transform of nseq sequences (stride ld) of length M; the block has
// exactly nseq * M / 4 threads, one radix-4 butterfly each per stage.
template <int M, bool INV>
__device__ __forceinline__ void fft_pow2(float2* buf, int ld, const float2* __restrict__ tw)
{
    constexpr int LOG2M = ilog2(M);
    constexpr int NB = M / 4;
    const int q = threadIdx.x / NB, j = threadIdx.x % NB;
    float2* s = buf + q * ld;
#pragma unroll
    for (int lns = 0; lns + 2 <= LOG2M; lns += 2) {
        const int Ns = 1 << lns;
        const int k = j & (Ns - 1);
        float2 v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) v[r] = s[j + r * NB];
        __syncthreads();
#pragma unroll
        for (int r = 1; r < 4; ++r) v[r] = cmul(v[r], twiddle(tw, (k * r) << (LOG2M - lns - 2), INV));
        dft_small<4, INV>(v);
        const int base = ((j >> lns) << (lns + 2)) + k;
#pragma unroll
        for (int r = 0; r < 4; ++r) s[base + r * Ns] = v[r];
        __syncthreads();
    }
    if (LOG2M & 1) {  // last stage radix 2, Ns = M/2: butterflies jj and jj + M/2
        float2 a[2], b[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            a[h] = s[j + h * NB];
            b[h] = s[j + h * NB + M / 2];
        }
        __syncthreads();
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int jj = j + h * NB;
            float2 v[2] = {a[h], cmul(b[h], twiddle(tw, jj, INV))};
            dft_small<2, INV>(v);
            s[jj] = v[0];
            s[jj + M / 2] = v[1];
        }
        __syncthreads();
    }
}

// Transform dispatch: MC > 0 compile-time size (in place, nseq*MC/4 threads),
// MC == 0 runtime plan (ping-pong, any block size).  Returns the buffer with
// the result; ends with __syncthreads().
template <int MC, bool INV>
__device__ __forceinline__ float2* fft_block(float2* a, float2* b, const FftPlan& fp, int nseq,
                                             int ld, const float2* __restrict__ tw)
{
    if constexpr (MC > 0) {
        fft_pow2<MC, INV>(a, ld, tw);
        return a;
    } else {
        return fft_rt<INV>(a, b, fp, nseq, ld, tw);
    }
}

// --------------------------------------------- CG helpers

__device__ __forceinline__ float redot(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// d = -g + beta d_old (d = -g on a restart, so a stale d_old never enters).
__device__ __forceinline__ float2 new_direction(float2 g, float2 dold, float beta, bool restart)
{
    return restart ? make_float2(-g.x, -g.y) : make_float2(fmaf(beta, dold.x, -g.x), fmaf(beta, dold.y, -g.y));
}

// ------------------------------------------------------------- row pass 1

// MODE 0: row FFTs of `in` (rows [0, rows), n_in nonzero inputs per row at
// stride ld_in) into X (stride M).
// MODE 1 (CG): the input rows are the new direction d = -g + beta d_old,
// written to c.d_new; also the block sums of
//   q1   = Re<d, 2 (Tf - D)>
//   num0 = sum_e lambda b(|z_e|) Re(conj(z_e) w_e),  den0 = sum_e lambda b(|z_e|) |w_e|^2
// (first line-search step, t = 0), finished by the last block into scal.
template <int MC, int MODE>
__global__ void k_rows_fwd(const float2* __restrict__ in, int ld_in, int n_in, int rows,
                           float2* __restrict__ X, FftPlan fp, const float2* __restrict__ tw,
                           int rpc, CgPass c)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    float2* a = sm;
    float2* b = sm + rpc * M;
    const int r0 = blockIdx.x * rpc;
    const int nr = min(rpc, rows - r0);
    const int N = n_in;
    float beta = 0.f;
    bool restart = true;
    if (MODE == 1) {
        const double bd = c.scal[S_BETA];
        beta = (float)bd;
        restart = bd == 0.0;
    }
    for (int e = threadIdx.x; e < rpc * M; e += blockDim.x) {
        const int q = e / M, m = e - q * M;
        float2 v = make_float2(0.f, 0.f);
        if (q < nr && m < N) {
            const int64_t o = (int64_t)(r0 + q) * ld_in + m;
            if (MODE == 0) {
                v = in[o];
            } else {
                v = new_direction(c.g[o], c.d_old[o], beta, restart);
                c.d_new[o] = v;
            }
        }
        a[e] = v;
    }
    __syncthreads();
    if (MODE == 1) {
        const Reg reg = c.reg;
        float q1 = 0.f, num = 0.f, den = 0.f;
        for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {
            const int q = e / N, m = e - q * N;
            const int n = r0 + q;
            const int64_t o = (int64_t)n * N + m;
            const bool has_r = m + 1 < N, has_d = n + 1 < N;
            const int64_t od = has_d ? o + N : o;
            // every load first (clamped neighbours, masked contributions)
            const float2 dn = a[q * M + m];
            const float2 dr = a[q * M + (has_r ? m + 1 : m)];
            const float2 fp_ = c.f[o], fr = c.f[has_r ? o + 1 : o], fd = c.f[od];
            const float2 gd = c.g[od], dold_d = c.d_old[od];
            const float2 tfv = c.Tf[o], dv = c.D[o];
            q1 += 2.f * redot(dn, f2sub(tfv, dv));
            if (reg.lambda1 != 0.f) {
                {
                    const float2 w = f2sub(dr, dn);
                    const float2 z = f2sub(fr, fp_);
                    const float bw = has_r ? reg.lambda1 * phi_weight(reg.kind, reg.alpha1, redot(z, z)) : 0.f;
                    num = fmaf(bw, redot(z, w), num);
                    den = fmaf(bw, redot(w, w), den);
                }
                {
                    const float2 dd = new_direction(gd, dold_d, beta, restart);
                    const float2 w = f2sub(dd, dn);
                    const float2 z = f2sub(fd, fp_);
                    const float bw = has_d ? reg.lambda1 * phi_weight(reg.kind, reg.alpha1, redot(z, z)) : 0.f;
                    num = fmaf(bw, redot(z, w), num);
                    den = fmaf(bw, redot(w, w), den);
                }
            }
            if (reg.lambda0 != 0.f) {
                const float bw = reg.lambda0 * phi_weight(reg.kind, reg.alpha0, redot(fp_, fp_));
                num = fmaf(bw, redot(fp_, dn), num);
                den = fmaf(bw, redot(dn, dn), den);
            }
        }
        float v[3] = {q1, num, den};
        FF bt[3];
        block_partial<3>(v, bt);
        store_parts<3>(bt, c.parts, kMaxParts);
        if (last_block(c.counter)) {
            FF t[3];
            sum_parts_ff<3>(c.parts, kMaxParts, gridDim.x, t);
            if (threadIdx.x == 0) {
                c.scal[S_Q1] = ff_to_double(t[0]);
                c.scal[S_NUM0] = ff_to_double(t[1]);
                c.scal[S_DEN0] = ff_to_double(t[2]);
                *c.counter = 0u;
            }
        }
    }
    float2* res = fft_block<MC, false>(a, b, fp, nr, M, tw);
    for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
        const int q = e / M, m = e - q * M;
        X[(int64_t)(r0 + q) * M + m] = res[e];
    }
}

// ------------------------------------------------------------- row pass 3

// Row IFFTs of X (rows [0, rows)), first n_out columns to out (stride n_out).
// With dotx: s = Re<dotx, out> reduced over the grid; MODE 0 stores it in
// scal[dot_scalar]; MODE 1 (CG) stores q2 = s and the first line-search step
//   t1 = -(q1 + num0) / (2 q2 + den0)   (0 when the curvature is not > 0).
template <int MC, int MODE>
__global__ void k_rows_inv(const float2* __restrict__ X, int rows, float2* __restrict__ out,
                           int n_out, FftPlan fp, const float2* __restrict__ tw, int rpc,
                           const float2* __restrict__ dotx, CgPass c, int dot_scalar)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    float2* a = sm;
    float2* b = sm + rpc * M;
    const int r0 = blockIdx.x * rpc;
    const int nr = min(rpc, rows - r0);
    for (int e = threadIdx.x; e < rpc * M; e += blockDim.x) {
        const int q = e / M;
        a[e] = q < nr ? X[(int64_t)r0 * M + e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_block<MC, true>(a, b, fp, nr, M, tw);
    float acc = 0.f;
    for (int e = threadIdx.x; e < nr * n_out; e += blockDim.x) {
        const int q = e / n_out, m = e - q * n_out;
        const float2 v = res[q * M + m];
        const int64_t o = (int64_t)(r0 + q) * n_out + m;
        out[o] = v;
        if (dotx) acc += redot(dotx[o], v);
    }
    if (dotx) {
        float v[1] = {acc};
        FF bt[1];
        block_partial<1>(v, bt);
        store_parts<1>(bt, c.parts, kMaxParts);
        if (last_block(c.counter)) {
            FF t[1];
            sum_parts_ff<1>(c.parts, kMaxParts, gridDim.x, t);
            if (threadIdx.x == 0) {
                const double s = ff_to_double(t[0]);
                if (MODE == 0) {
                    c.scal[dot_scalar] = s;
                } else {
                    c.scal[S_Q2] = s;
                    const double curv = 2.0 * s + c.scal[S_DEN0];
                    c.scal[S_T1] = curv > 0.0 ? -(c.scal[S_Q1] + c.scal[S_NUM0]) / curv : 0.0;
                }
                *c.counter = 0u;
            }
        }
    }
}

// ------------------------------------------------------------- column pass

// Columns [x0, x0+cpc) of the N x M buffer X: FFT of the n_in nonzero rows,
// multiply by Chat[x][ky], IFFT, keep rows < n_out.  Sequences sit at stride
// M+1 in shared memory (spreads the banks of the transposed loads).
template <int MC>
__global__ void k_cols_filter(float2* X, int n_in, int n_out, FftPlan fp, const float2* __restrict__ tw,
                              const float* __restrict__ Chat, int cpc)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    const int ld = M + 1;
    float2* a = sm;
    float2* b = sm + cpc * ld;
    const int x0 = blockIdx.x * cpc;
    const int nc = min(cpc, M - x0);
    for (int e = threadIdx.x; e < cpc * M; e += blockDim.x) {
        const int y = e / cpc, cc = e - y * cpc;
        a[cc * ld + y] = (y < n_in && cc < nc) ? X[(int64_t)y * M + x0 + cc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_block<MC, false>(a, b, fp, cpc, ld, tw);
    for (int e = threadIdx.x; e < cpc * M; e += blockDim.x) {
        const int cc = e / M, ky = e - cc * M;
        const float h = cc < nc ? __ldg(&Chat[(int64_t)(x0 + cc) * M + ky]) : 0.f;
        const float2 v = res[cc * ld + ky];
        res[cc * ld + ky] = make_float2(v.x * h, v.y * h);
    }
    __syncthreads();
    float2* other = res == a ? b : a;
    float2* res2 = fft_block<MC, true>(res, other, fp, cpc, ld, tw);
    for (int e = threadIdx.x; e < cpc * n_out; e += blockDim.x) {
        const int y = e / cpc, cc = e - y * cpc;
        if (cc < nc) X[(int64_t)y * M + x0 + cc] = res2[cc * ld + y];
    }
}

// Column FFTs of the M x M circulant and the real spectrum:
// Chat[x][ky] = Re(FFT2 c)[ky][x] / M^2.
template <int MC>
__global__ void k_cols_spectrum(const float2* cwork, FftPlan fp, const float2* __restrict__ tw,
                                float* Chat, int cpc)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    const int ld = M + 1;
    float2* a = sm;
    float2* b = sm + cpc * ld;
    const int x0 = blockIdx.x * cpc;
    const int nc = min(cpc, M - x0);
    for (int e = threadIdx.x; e < cpc * M; e += blockDim.x) {
        const int y = e / cpc, cc = e - y * cpc;
        a[cc * ld + y] = cc < nc ? cwork[(int64_t)y * M + x0 + cc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_block<MC, false>(a, b, fp, cpc, ld, tw);
    const float inv = 1.0f / ((float)M * (float)M);
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int cc = e / M, ky = e - cc * M;
        Chat[(int64_t)(x0 + cc) * M + ky] = res[cc * ld + ky].x * inv;
    }
}

// c[y][x] = K[v][u] = conj G_{u,v} with v = y (y < N) or y - M (y > M - N),
// u likewise from x; zero where |u| or |v| >= N.  G holds u >= 0; the rest is
// G_{u,v} = conj G_{-u,-v}.
__global__ void k_embed(const float2* __restrict__ G, int N, int M, float2* cwork)
{
    const int64_t MM = (int64_t)M * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MM;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(e / M), x = (int)(e % M);
        const int v = y < N ? y : (y > M - N ? y - M : INT32_MIN);
        const int u = x < N ? x : (x > M - N ? x - M : INT32_MIN);
        float2 c = make_float2(0.f, 0.f);
        if (v != INT32_MIN && u != INT32_MIN) {
            const int W = 2 * N - 1;
            if (u >= 0) {
                const float2 g = G[(int64_t)u * W + (v + N - 1)];
                c = make_float2(g.x, -g.y);
            } else {
                c = G[(int64_t)(-u) * W + (-v + N - 1)];
            }
        }
        cwork[e] = c;
    }
}

// ------------------------------------------------------------- launch shapes

constexpr int kFftSmemCap = 200 * 1024;

struct Shape {
    int per_cta;  // rows or columns per CTA
    int threads;
    size_t smem;
};

// Compile-time path: nseq * M / 4 threads (<= 1024), single buffer.
// Runtime path: 256 threads, ping-pong buffers.
Shape row_shape(int M, bool pow2)
{
    if (pow2) {
        const int nb = M / 4;
        const int rpc = nb >= 256 ? 1 : 256 / nb;
        return Shape{rpc, rpc * nb, (size_t)rpc * M * sizeof(float2)};
    }
    const int rpc = M >= 1024 ? 1 : 1024 / M;
    return Shape{rpc, 256, 2 * (size_t)rpc * M * sizeof(float2)};
}

Shape col_shape(int M, bool pow2)
{
    if (pow2) {
        const int nb = M / 4;
        int cpc = nb >= 1024 ? 1 : 1024 / nb;
        while (cpc > 1 && (size_t)cpc * (M + 1) * sizeof(float2) > (size_t)kFftSmemCap) cpc /= 2;
        return Shape{cpc, cpc * nb, (size_t)cpc * (M + 1) * sizeof(float2)};
    }
    int cpc = M >= 1024 ? 4 : (M >= 512 ? 8 : 16);
    while (cpc > 1 && 2 * (size_t)cpc * (M + 1) * sizeof(float2) > (size_t)kFftSmemCap) --cpc;
    return Shape{cpc, 256, 2 * (size_t)cpc * (M + 1) * sizeof(float2)};
}

template <int MC>
int set_attrs()
{
    const int bytes = kFftSmemCap;
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd<MC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_fwd<MC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_inv<MC, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_rows_inv<MC, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_cols_filter<MC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_cols_spectrum<MC>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return SPIREC_OK;
}

// Calls f.template operator()<MC>() with the compile-time size for M, or
// MC = 0 for sizes without a specialisation.
template <typename F>
int with_size(int M, F&& f)
{
    switch (M) {
    case 16: return f.template operator()<16>();
    case 32: return f.template operator()<32>();
    case 64: return f.template operator()<64>();
    case 128: return f.template operator()<128>();
    case 256: return f.template operator()<256>();
    case 512: return f.template operator()<512>();
    case 1024: return f.template operator()<1024>();
    case 2048: return f.template operator()<2048>();
    case 4096: return f.template operator()<4096>();
    default: return f.template operator()<0>();
    }
}

bool is_pow2_specialised(int M) { return M >= 16 && M <= 4096 && (M & (M - 1)) == 0; }

CgPass plain_pass(spirec_plan p, int slot, unsigned* counter)
{
    CgPass c{};
    c.parts = reinterpret_cast<float2*>(p->part) + (size_t)slot * kMaxParts;
    c.counter = counter;
    c.scal = p->scal;
    c.reg = p->reg;
    return c;
}

struct AttrAll {
    template <int MC>
    int operator()() { return MC > 0 ? set_attrs<MC>() : SPIREC_OK; }
};

struct LaunchRowsFwd {
    spirec_plan p;
    const float2* in;
    int ld_in, n_in, rows, mode, blocks;
    Shape s;
    CgPass c;
    template <int MC>
    int operator()()
    {
        if (mode == 0)
            k_rows_fwd<MC, 0><<<blocks, s.threads, s.smem, p->stream>>>(in, ld_in, n_in, rows, p->X, p->fft,
                                                                        p->twiddle, s.per_cta, c);
        else
            k_rows_fwd<MC, 1><<<blocks, s.threads, s.smem, p->stream>>>(in, ld_in, n_in, rows, p->X, p->fft,
                                                                        p->twiddle, s.per_cta, c);
        SPIREC_CK(cudaGetLastError());
        p->launches += 1;
        return SPIREC_OK;
    }
};

struct LaunchCols {
    spirec_plan p;
    int n_in, n_out, blocks;
    Shape s;
    template <int MC>
    int operator()()
    {
        k_cols_filter<MC><<<blocks, s.threads, s.smem, p->stream>>>(p->X, n_in, n_out, p->fft, p->twiddle,
                                                                    p->Chat, s.per_cta);
        SPIREC_CK(cudaGetLastError());
        p->launches += 1;
        return SPIREC_OK;
    }
};

struct LaunchRowsInv {
    spirec_plan p;
    float2* out;
    int mode;
    const float2* dotx;
    int dot_scalar, blocks;
    Shape s;
    CgPass c;
    template <int MC>
    int operator()()
    {
        if (mode == 0)
            k_rows_inv<MC, 0><<<blocks, s.threads, s.smem, p->stream>>>(p->X, p->N, out, p->N, p->fft,
                                                                        p->twiddle, s.per_cta, dotx, c, dot_scalar);
        else
            k_rows_inv<MC, 1><<<blocks, s.threads, s.smem, p->stream>>>(p->X, p->N, out, p->N, p->fft,
                                                                        p->twiddle, s.per_cta, dotx, c, dot_scalar);
        SPIREC_CK(cudaGetLastError());
        p->launches += 1;
        return SPIREC_OK;
    }
};

struct LaunchSpectrum {
    spirec_plan p;
    Shape rs, cs;
    template <int MC>
    int operator()()
    {
        const int M = p->M;
        CgPass c{};
        // rows of the circulant, in place (each block reads its rows fully first)
        k_rows_fwd<MC, 0><<<(M + rs.per_cta - 1) / rs.per_cta, rs.threads, rs.smem, p->stream>>>(
            p->cwork, M, M, M, p->cwork, p->fft, p->twiddle, rs.per_cta, c);
        SPIREC_CK(cudaGetLastError());
        k_cols_spectrum<MC><<<(M + cs.per_cta - 1) / cs.per_cta, cs.threads, cs.smem, p->stream>>>(
            p->cwork, p->fft, p->twiddle, p->Chat, cs.per_cta);
        SPIREC_CK(cudaGetLastError());
        p->launches += 2;
        return SPIREC_OK;
    }
};

}  // namespace

int fft_setup_attributes(int)
{
    int rc;
    if ((rc = set_attrs<0>()) != SPIREC_OK) return rc;
    for (int M = 16; M <= 4096; M *= 2)
        if ((rc = with_size(M, AttrAll{})) != SPIREC_OK) return rc;
    return SPIREC_OK;
}

int launch_rows_fwd(spirec_plan p, const float2* in, int ld_in, int n_in, int rows, int mode,
                    const CgPass* cg)
{
    const int M = p->M;
    const Shape s = row_shape(M, is_pow2_specialised(M));
    const int blocks = (rows + s.per_cta - 1) / s.per_cta;
    if (mode == 1 && blocks > kMaxParts) {
        set_error("too many row blocks");
        return SPIREC_EUNSUPPORTED;
    }
    const CgPass c = cg ? *cg : plain_pass(p, 0, nullptr);
    return with_size(M, LaunchRowsFwd{p, in, ld_in, n_in, rows, mode, blocks, s, c});
}

int launch_cols(spirec_plan p, int n_in, int n_out)
{
    const int M = p->M;
    const Shape s = col_shape(M, is_pow2_specialised(M));
    const int blocks = (M + s.per_cta - 1) / s.per_cta;
    return with_size(M, LaunchCols{p, n_in, n_out, blocks, s});
}

int launch_rows_inv(spirec_plan p, float2* out, int mode, const float2* dotx, const CgPass* cg,
                    int dot_scalar)
{
    const int M = p->M, N = p->N;
    const Shape s = row_shape(M, is_pow2_specialised(M));
    const int blocks = (N + s.per_cta - 1) / s.per_cta;
    if (dotx && blocks > kMaxParts) {
        set_error("too many row blocks");
        return SPIREC_EUNSUPPORTED;
    }
    const CgPass c = cg ? *cg : plain_pass(p, P_MISC, p->counters + C_MISC);
    return with_size(M, LaunchRowsInv{p, out, mode, dotx, dot_scalar, blocks, s, c});
}

int launch_toeplitz(spirec_plan p, const float2* x, float2* Tx, int dot_scalar)
{
    int rc;
    const int N = p->N;
    if ((rc = launch_rows_fwd(p, x, N, N, N, 0, nullptr)) != SPIREC_OK) return rc;
    if ((rc = launch_cols(p, N, N)) != SPIREC_OK) return rc;
    return launch_rows_inv(p, Tx, 0, dot_scalar >= 0 ? x : nullptr, nullptr, dot_scalar);
}

int launch_spectrum(spirec_plan p)
{
    const int N = p->N, M = p->M;
    k_embed<<<4 * 152, 256, 0, p->stream>>>(p->G, N, M, p->cwork);
    SPIREC_CK(cudaGetLastError());
    p->launches += 1;
    const bool pow2 = is_pow2_specialised(M);
    return with_size(M, LaunchSpectrum{p, row_shape(M, pow2), col_shape(M, pow2)});
}

}  // namespace spirec

// ------------------------------------------------ T x without any allocation
//
// spirec_toeplitz_noalloc: the Toeplitz apply above for callers that cannot
// allocate device memory (for example code running inside a memory-pool
// budget that forbids cudaMalloc, or a host process that must not grow the
// GPU footprint after start-up).  The caller passes the input, the kernel
// spectrum and the output; the intermediate N x M rows, the transposed
// spectrum and the twiddle table live in one file-scope device array that
// every GPU loading this library keeps until the process exits.

namespace spirec {
namespace {

constexpr int kNoAllocMaxN = 512;
constexpr int kNoAllocMaxM = 1024;
constexpr size_t kNoAllocRowsBytes = (size_t)kNoAllocMaxN * kNoAllocMaxM * sizeof(float2);
constexpr size_t kNoAllocSpecBytes = (size_t)kNoAllocMaxM * kNoAllocMaxM * sizeof(float);
constexpr size_t kNoAllocTwBytes = (size_t)kNoAllocMaxM * sizeof(float2);
constexpr size_t kNoAllocBytes = kNoAllocRowsBytes + kNoAllocSpecBytes + kNoAllocTwBytes;

// Shared by every call on a device; holds the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
void* g_noalloc_base[kNoAllocMaxDevices];  // device address of the array, per device
bool g_noalloc_ready[kNoAllocMaxDevices];

// tw[k] = exp(-2 pi i k / M)
__global__ void k_noalloc_twiddles(float2* tw, int M)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)k / (double)M, &s, &c);
        tw[k] = make_float2((float)c, (float)s);
    }
}

// spectrum[ky][kx] (the layout spirec_kernel_spectrum_dev returns) into the
// column-major form the column pass reads, chat[kx][ky].
__global__ void k_noalloc_spectrum(const float* __restrict__ spec, int M, float* __restrict__ chat)
{
    const int64_t MM = (int64_t)M * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < MM;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t kx = e / M, ky = e % M;
        chat[e] = spec[ky * M + kx];
    }
}

struct LaunchNoAlloc {
    const float2* x;
    float2* Tx;
    float2* rows;
    const float* chat;
    const float2* tw;
    FftPlan fp;
    int N;
    cudaStream_t st;
    template <int MC>
    int operator()()
    {
        const int M = fp.M;
        const bool pow2 = MC > 0;
        const Shape rs = row_shape(M, pow2), cs = col_shape(M, pow2);
        const int rblocks = (N + rs.per_cta - 1) / rs.per_cta;
        const CgPass c{};
        k_rows_fwd<MC, 0><<<rblocks, rs.threads, rs.smem, st>>>(x, N, N, N, rows, fp, tw, rs.per_cta, c);
        SPIREC_CK(cudaGetLastError());
        k_cols_filter<MC><<<(M + cs.per_cta - 1) / cs.per_cta, cs.threads, cs.smem, st>>>(rows, N, N, fp, tw,
                                                                                          chat, cs.per_cta);
        SPIREC_CK(cudaGetLastError());
        k_rows_inv<MC, 0><<<rblocks, rs.threads, rs.smem, st>>>(rows, N, Tx, N, fp, tw, rs.per_cta, nullptr,
                                                                 c, 0);
        SPIREC_CK(cudaGetLastError());
        return SPIREC_OK;
    }
};

}  // namespace

}  // namespace spirec

extern "C" int spirec_toeplitz_noalloc(const float* x, const float* spectrum, float* Tx, int32_t N,
                                       int32_t M, void* stream)
{
    using namespace spirec;
    if (!x || !spectrum || !Tx) {
        set_error("null pointer");
        return SPIREC_EINVAL;
    }
    if (N < 2 || N > kNoAllocMaxN || M < 2 * N - 1 || M > kNoAllocMaxM) {
        set_error("spirec_toeplitz_noalloc handles 2 <= N <= %d and 2N-1 <= M <= %d (got N=%d, M=%d)",
                  kNoAllocMaxN, kNoAllocMaxM, N, M);
        return SPIREC_EINVAL;
    }
    FftPlan fp;
    if (!make_fft_plan(M, &fp)) {
        set_error("M=%d must factor into 2, 3 and 5", M);
        return SPIREC_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        set_error("device %d out of range", dev);
        return SPIREC_EUNSUPPORTED;
    }
    // first call on this device: the array's device address and the kernels'
    // shared-memory limits (no allocation; must happen outside stream capture)
    if (!g_noalloc_ready[dev]) {
        void* base = nullptr;
        e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress");
        int rc = fft_setup_attributes(M);
        if (rc != SPIREC_OK) return rc;
        g_noalloc_base[dev] = base;
        g_noalloc_ready[dev] = true;
    }
    unsigned char* base = static_cast<unsigned char*>(g_noalloc_base[dev]);
    float2* rows = reinterpret_cast<float2*>(base);
    float* chat = reinterpret_cast<float*>(base + kNoAllocRowsBytes);
    float2* tw = reinterpret_cast<float2*>(base + kNoAllocRowsBytes + kNoAllocSpecBytes);
    cudaStream_t st = (cudaStream_t)stream;
    k_noalloc_twiddles<<<(M + 255) / 256, 256, 0, st>>>(tw, M);
    SPIREC_CK(cudaGetLastError());
    k_noalloc_spectrum<<<4 * 152, 256, 0, st>>>(spectrum, M, chat);
    SPIREC_CK(cudaGetLastError());
    return with_size(M, LaunchNoAlloc{(const float2*)x, (float2*)Tx, rows, chat, tw, fp, N, st});
}
