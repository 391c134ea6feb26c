// fft_device.cuh -- device code of the Toeplitz apply (see fft.cu for the
// math): shared-memory Stockham FFTs and the per-group bodies of the three
// passes, including the CG work fused into the row passes.  Used by the
// stand-alone pass kernels (fft.cu) and by the persistent CG loop
// (cg_loop.cu).
//
// Buffers written inside a persistent kernel by other blocks (the row buffer
// X, the iterates) are read with ld.global.cg (L2, never a stale L1 line).
#pragma once

#include <stdint.h>

#include "internal.cuh"
#include "phase.cuh"

namespace spirec {
namespace fftd {

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

// Twiddle e of the table; TWS: the table is in shared memory (a plain
// load), else in global memory (read-only path).
template <bool TWS = false>
__device__ __forceinline__ float2 twiddle(const float2* __restrict__ tw, int e, bool inv)
{
    float2 w = TWS ? tw[e] : __ldg(tw + e);
    if (inv) w.y = -w.y;
    return w;
}

// Shared-memory index of element i of a sequence: the compile-time path
// inserts one slot every 16 elements (spreads the strided Stockham stores
// over the banks); the runtime path stores densely.
template <int MC>
__device__ __forceinline__ int sidx(int i)
{
    return MC > 0 ? i + (i >> 4) : i;
}
template <int MC>
__host__ __device__ constexpr int seq_len(int M)
{
    return MC > 0 ? M + (M >> 4) : M;
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

// Staged twiddle table (shared memory) for fft_pow2 of size M: the radix-4
// stage with span Ns keeps w^((k r) M / (4 Ns)) at (Ns - 1) + (r - 1) Ns + k
// (r = 1..3, k < Ns), so the lanes of a warp, which hold consecutive k, read
// consecutive entries or the same one (no bank conflicts); the radix-2 stage
// of an odd log2 M keeps w^jj at r4_entries + jj.  From the plain table
// tw[e] = w^e.  Entries: staged_twiddles_size(M) <= 3M/2.
__host__ __device__ constexpr int staged_r4_entries(int M) { return (1 << (2 * (ilog2(M) / 2))) - 1; }
__host__ __device__ constexpr int staged_twiddles_size(int M)
{
    return staged_r4_entries(M) + ((ilog2(M) & 1) ? M / 2 : 0);
}
template <int M>
__device__ __forceinline__ void build_staged_twiddles(const float2* __restrict__ tw, float2* stw)
{
    constexpr int LOG2M = ilog2(M);
    for (int lns = 0; lns + 2 <= LOG2M; lns += 2) {
        const int Ns = 1 << lns;
        for (int i = threadIdx.x; i < 3 * Ns; i += blockDim.x) {
            const int r = i / Ns + 1, k = i - (r - 1) * Ns;
            stw[Ns - 1 + i] = __ldg(tw + ((k * r) << (LOG2M - lns - 2)));
        }
    }
    if (LOG2M & 1)
        for (int jj = threadIdx.x; jj < M / 2; jj += blockDim.x) stw[staged_r4_entries(M) + jj] = __ldg(tw + jj);
}

// In-place transform of BPT * blockDim.x / (M/4) sequences (stride ld,
// padded index) of length M: BPT radix-4 butterflies per thread per stage
// (plus one radix-2 stage for odd log2 M), values held in registers between
// a read and a write phase.  TWS: tw is the staged table in shared memory
// (build_staged_twiddles), else the plain table in global memory.
template <int M, bool INV, int BPT = 1, bool TWS = false>
__device__ __forceinline__ void fft_pow2(float2* buf, int ld, const float2* __restrict__ tw)
{
    constexpr int LOG2M = ilog2(M);
    constexpr int NB = M / 4;
    const int q0 = threadIdx.x / NB, j = threadIdx.x % NB;
    const int qstep = blockDim.x / NB;
#pragma unroll
    for (int lns = 0; lns + 2 <= LOG2M; lns += 2) {
        const int Ns = 1 << lns;
        const int k = j & (Ns - 1);
        float2 v[BPT][4];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const float2* s = buf + (q0 + b * qstep) * ld;
#pragma unroll
            for (int r = 0; r < 4; ++r) v[b][r] = s[sidx<M>(j + r * NB)];
        }
        __syncthreads();
        float2 w[4];
#pragma unroll
        for (int r = 1; r < 4; ++r)
            w[r] = TWS ? twiddle<true>(tw, Ns - 1 + (r - 1) * Ns + k, INV)
                       : twiddle<false>(tw, (k * r) << (LOG2M - lns - 2), INV);
        const int base = ((j >> lns) << (lns + 2)) + k;
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
#pragma unroll
            for (int r = 1; r < 4; ++r) v[b][r] = cmul(v[b][r], w[r]);
            dft_small<4, INV>(v[b]);
            float2* s = buf + (q0 + b * qstep) * ld;
#pragma unroll
            for (int r = 0; r < 4; ++r) s[sidx<M>(base + r * Ns)] = v[b][r];
        }
        __syncthreads();
    }
    if (LOG2M & 1) {  // last stage radix 2, Ns = M/2: butterflies jj and jj + M/2
        float2 a[BPT][2], c[BPT][2];
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            const float2* s = buf + (q0 + b * qstep) * ld;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                a[b][h] = s[sidx<M>(j + h * NB)];
                c[b][h] = s[sidx<M>(j + h * NB + M / 2)];
            }
        }
        __syncthreads();
#pragma unroll
        for (int b = 0; b < BPT; ++b) {
            float2* s = buf + (q0 + b * qstep) * ld;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int jj = j + h * NB;
                float2 v[2] = {a[b][h],
                               cmul(c[b][h], twiddle<TWS>(tw, TWS ? staged_r4_entries(M) + jj : jj, INV))};
                dft_small<2, INV>(v);
                s[sidx<M>(jj)] = v[0];
                s[sidx<M>(jj + M / 2)] = v[1];
            }
        }
        __syncthreads();
    }
}

// MC > 0: compile-time size, in place, blockDim.x * BPT = nseq * MC / 4.
// MC == 0: runtime plan, ping-pong, any block size.  Returns the buffer with
// the result; ends with __syncthreads().
template <int MC, bool INV, int BPT = 1>
__device__ __forceinline__ float2* fft_block(float2* a, float2* b, const FftPlan& fp, int nseq,
                                             int ld, const float2* __restrict__ tw)
{
    if constexpr (MC > 0) {
        fft_pow2<MC, INV, BPT>(a, ld, tw);
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

// ------------------------------------------------------ row pass 1, a group

// Rows [r0, r0 + rpc) (nr of them real).  MODE 0: the rows of `in` (n_in
// nonzero entries, stride ld_in).  MODE 1 (CG): the rows of the new direction
// d = -g + beta d_old, written to c.d_new, with the per-thread sums
//   acc[0] += Re<d, 2 res>, res = T f - D             (q1)
//   acc[1] += sum_e lambda b(|z_e|) Re(conj(z_e) w_e)  (h'(0) penalty part)
//   acc[2] += sum_e lambda b(|z_e|) |w_e|^2            (curvature at t = 0)
// over the right/down edges and pixels of these rows.  Then the FFTs and the
// M outputs of each row into X.
template <int MC, int MODE, int KIND = -1>
__device__ __forceinline__ void rows_fwd_group(const float2* in, int ld_in, int n_in, int r0, int nr,
                                               int rpc, float2* X, const FftPlan& fp,
                                               const float2* __restrict__ tw, const CgPass& c,
                                               float beta, bool restart, float2* a, float2* b,
                                               float (&acc)[3])
{
    const int M = fp.M;
    const int ld = seq_len<MC>(M);
    const int N = n_in;
    if constexpr (MC > 0) {
        // rpc * M == 4 * blockDim.x: four elements per thread, loads first
        float2 ga[4], gb[4];
        bool live[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = threadIdx.x + i * blockDim.x;
            const int q = e / M, m = e - q * M;
            live[i] = q < nr && m < N;
            const int64_t o = live[i] ? (int64_t)(r0 + q) * ld_in + m : 0;
            if (MODE == 0) {
                ga[i] = live[i] ? __ldcg(in + o) : make_float2(0.f, 0.f);
            } else {
                ga[i] = live[i] ? __ldcg(c.g + o) : make_float2(0.f, 0.f);
                gb[i] = live[i] ? __ldcg(c.d_old + o) : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = threadIdx.x + i * blockDim.x;
            const int q = e / M, m = e - q * M;
            float2 v = make_float2(0.f, 0.f);
            if (live[i]) {
                if (MODE == 0) {
                    v = ga[i];
                } else {
                    v = new_direction(ga[i], gb[i], beta, restart);
                    c.d_new[(int64_t)(r0 + q) * ld_in + m] = v;
                }
            }
            a[q * ld + sidx<MC>(m)] = v;
        }
    } else {
        for (int e = threadIdx.x; e < rpc * M; e += blockDim.x) {
            const int q = e / M, m = e - q * M;
            float2 v = make_float2(0.f, 0.f);
            if (q < nr && m < N) {
                const int64_t o = (int64_t)(r0 + q) * ld_in + m;
                if (MODE == 0) {
                    v = __ldcg(in + o);
                } else {
                    v = new_direction(__ldcg(c.g + o), __ldcg(c.d_old + o), beta, restart);
                    c.d_new[o] = v;
                }
            }
            a[q * ld + sidx<MC>(m)] = v;
        }
    }
    __syncthreads();
    if (MODE == 1) {
        const Reg reg = c.reg;
#pragma unroll 2
        for (int e = threadIdx.x; e < nr * N; e += blockDim.x) {            const int q = e / N, m = e - q * N;
            const int n = r0 + q;
            const int64_t o = (int64_t)n * N + m;
            const bool has_r = m + 1 < N, has_d = n + 1 < N;
            const int64_t od = has_d ? o + N : o;
            // every load first (clamped neighbours, masked contributions)
            const float2 dn = a[q * ld + sidx<MC>(m)];
            const float2 dr = a[q * ld + sidx<MC>(has_r ? m + 1 : m)];
            const float2 fp_ = __ldcg(c.f + o), fr = __ldcg(c.f + (has_r ? o + 1 : o)), fd = __ldcg(c.f + od);
            const float2 gd = __ldcg(c.g + od), dold_d = __ldcg(c.d_old + od);
            acc[0] += 2.f * redot(dn, __ldcg(c.res + o));
            if (reg.lambda1 != 0.f) {
                {
                    const float2 w = f2sub(dr, dn);
                    const float2 z = f2sub(fr, fp_);
                    const float bw = has_r ? reg.lambda1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, redot(z, z)) : 0.f;
                    acc[1] = fmaf(bw, redot(z, w), acc[1]);
                    acc[2] = fmaf(bw, redot(w, w), acc[2]);
                }
                {
                    const float2 dd = new_direction(gd, dold_d, beta, restart);
                    const float2 w = f2sub(dd, dn);
                    const float2 z = f2sub(fd, fp_);
                    const float bw = has_d ? reg.lambda1 * phi_weight_k<KIND>(reg.kind, reg.alpha1, redot(z, z)) : 0.f;
                    acc[1] = fmaf(bw, redot(z, w), acc[1]);
                    acc[2] = fmaf(bw, redot(w, w), acc[2]);
                }
            }
            if (reg.lambda0 != 0.f) {
                const float bw = reg.lambda0 * phi_weight_k<KIND>(reg.kind, reg.alpha0, redot(fp_, fp_));
                acc[1] = fmaf(bw, redot(fp_, dn), acc[1]);
                acc[2] = fmaf(bw, redot(dn, dn), acc[2]);
            }
        }
    }
    float2* res = fft_block<MC, false>(a, b, fp, rpc, ld, tw);
    for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
        const int q = e / M, m = e - q * M;
        X[(int64_t)(r0 + q) * M + m] = res[q * ld + sidx<MC>(m)];
    }
}

// ------------------------------------------------------ row pass 3, a group

// Row IFFTs of X rows [r0, r0 + nr), first n_out columns to out (stride
// n_out); with dotx, acc += Re<dotx, out> over them.
template <int MC>
__device__ __forceinline__ void rows_inv_group(const float2* X, int r0, int nr, int rpc,
                                               float2* out, int n_out, const FftPlan& fp,
                                               const float2* __restrict__ tw, const float2* dotx,
                                               float2* a, float2* b, float& acc)
{
    const int M = fp.M;
    const int ld = seq_len<MC>(M);
    if constexpr (MC > 0) {
        float2 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = threadIdx.x + i * blockDim.x;
            const int q = e / M;
            v[i] = q < nr ? __ldcg(X + (int64_t)(r0 + q) * M + (e - q * M)) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = threadIdx.x + i * blockDim.x;
            const int q = e / M;
            a[q * ld + sidx<MC>(e - q * M)] = v[i];
        }
    } else {
        for (int e = threadIdx.x; e < rpc * M; e += blockDim.x) {
            const int q = e / M, m = e - q * M;
            a[q * ld + sidx<MC>(m)] = q < nr ? __ldcg(X + (int64_t)(r0 + q) * M + m) : make_float2(0.f, 0.f);
        }
    }
    __syncthreads();
    float2* res = fft_block<MC, true>(a, b, fp, rpc, ld, tw);
#pragma unroll 2
    for (int e = threadIdx.x; e < nr * n_out; e += blockDim.x) {        const int q = e / n_out, m = e - q * n_out;
        const float2 v = res[q * ld + sidx<MC>(m)];
        const int64_t o = (int64_t)(r0 + q) * n_out + m;
        out[o] = v;
        if (dotx) acc += redot(__ldcg(dotx + o), v);
    }
}

// ------------------------------------------------------ column pass, a group

// Columns [x0, x0 + nc) of the buffer X (M columns): FFT of the n_in nonzero
// rows, times Chat[x][ky], IFFT, rows < n_out back into X.  Sequences sit at
// stride seq_len + 4 (spreads the banks of the transposed loads).
// MODE 1 (the persistent CG loop, compile-time M only): the twiddle table is
// in shared memory and Chat is read through L2 only.
template <int MC, int BPT = 1, int MODE = 0>
__device__ __forceinline__ void cols_group(float2* X, int n_in, int n_out, int x0, int nc, int cpc,
                                           const FftPlan& fp, const float2* __restrict__ tw,
                                           const float* __restrict__ Chat, float2* a, float2* b)
{
    static_assert(MODE == 0 || MC > 0, "the CG column mode needs a compile-time size");
    const int M = fp.M;
    const int ld = seq_len<MC>(M) + 4;
    float2* res;
    if constexpr (MC > 0) {
        // cpc * M == 4 * BPT * blockDim.x: the column values and this thread's
        // spectrum values are all requested before the first is used
        constexpr int E = 4 * BPT;
        float2 v[E];
        float h[E];
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int e = threadIdx.x + i * blockDim.x;
            const int y = e / cpc, cc = e - y * cpc;
            const bool in = y < n_in && cc < nc;
            v[i] = in ? __ldcg(X + (int64_t)y * M + x0 + cc) : make_float2(0.f, 0.f);
            const int hc = e / M, hk = e - hc * M;
            h[i] = hc < nc ? (MODE == 1 ? __ldcg(&Chat[(int64_t)(x0 + hc) * M + hk])
                                        : __ldg(&Chat[(int64_t)(x0 + hc) * M + hk]))
                           : 0.f;
        }
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int e = threadIdx.x + i * blockDim.x;
            const int y = e / cpc, cc = e - y * cpc;
            a[cc * ld + sidx<MC>(y)] = v[i];
        }
        __syncthreads();
        fft_pow2<MC, false, BPT, MODE == 1>(a, ld, tw);
        res = a;
#pragma unroll
        for (int i = 0; i < E; ++i) {
            const int e = threadIdx.x + i * blockDim.x;
            const int cc = e / M, ky = e - cc * M;
            const int j = cc * ld + sidx<MC>(ky);
            const float2 x = res[j];
            res[j] = make_float2(x.x * h[i], x.y * h[i]);
        }
    } else {
        for (int e = threadIdx.x; e < cpc * M; e += blockDim.x) {
            const int y = e / cpc, cc = e - y * cpc;
            a[cc * ld + sidx<MC>(y)] =
                (y < n_in && cc < nc) ? __ldcg(X + (int64_t)y * M + x0 + cc) : make_float2(0.f, 0.f);
        }
        __syncthreads();
        res = fft_block<MC, false>(a, b, fp, cpc, ld, tw);
        for (int e = threadIdx.x; e < cpc * M; e += blockDim.x) {
            const int cc = e / M, ky = e - cc * M;
            const float hv = cc < nc ? __ldg(&Chat[(int64_t)(x0 + cc) * M + ky]) : 0.f;
            const int i = cc * ld + sidx<MC>(ky);
            const float2 x = res[i];
            res[i] = make_float2(x.x * hv, x.y * hv);
        }
    }
    __syncthreads();
    float2* other = res == a ? b : a;
    float2* res2;
    if constexpr (MC > 0) {
        fft_pow2<MC, true, BPT, MODE == 1>(res, ld, tw);
        res2 = res;
    } else {
        res2 = fft_block<MC, true, BPT>(res, other, fp, cpc, ld, tw);
    }
    for (int e = threadIdx.x; e < cpc * n_out; e += blockDim.x) {
        const int y = e / cpc, cc = e - y * cpc;
        if (cc < nc) X[(int64_t)y * M + x0 + cc] = res2[cc * ld + sidx<MC>(y)];
    }
}

}  // namespace fftd
}  // namespace spirec
