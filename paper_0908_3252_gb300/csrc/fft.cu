// fft.cu -- shared-memory mixed-radix FFTs for the Toeplitz (Gram) operator
// and its kernel spectrum.
//
// T x = H^H H x is a 2-D linear convolution of x with conj(G) (Appendix B).
// Embedded in an M x M circulant (M >= 2N-1, section 3.4's "circular
// convolution" after zero padding) it becomes
//     T x = crop_N( IFFT2( Chat .* FFT2( pad_M(x) ) ) ),
// with Chat = FFT2(c) / M^2 real because c[-y][-x] = conj c[y][x] (the point
// symmetry of G).  The apply runs in three passes over an N x M buffer:
//   1. N row FFTs of the zero-padded rows (N inputs, M outputs),
//   2. per column: FFT (N nonzero inputs) -> * Chat -> IFFT, keep rows < N,
//   3. N row IFFTs, keep columns < N, and the dot Re<x, T x> in FP64.
// Each FFT is a self-sorting Stockham transform in shared memory with radix
// 2, 3, 4 or 5 stages and a twiddle table exp(-2 pi i k / M).
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

// Small DFT of size R: X[q] = sum_r v[r] w^(r q), w = exp(-+2 pi i / R).
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
        // forward: X1 = s1 - i s3, X3 = s1 + i s3; inverse swaps them
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
        // s1 * i * u = (-s1 u.y, s1 u.x)
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
        // i * (s1 d1 + s2 d2) and i * (s2 d1 - s1 d2)
        const float2 e1 = make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y);
        const float2 e2 = make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y);
        v[1] = make_float2(m1.x - e1.y, m1.y + e1.x);
        v[4] = make_float2(m1.x + e1.y, m1.y - e1.x);
        v[2] = make_float2(m2.x - e2.y, m2.y + e2.x);
        v[3] = make_float2(m2.x + e2.y, m2.y - e2.x);
    }
}

// One Stockham stage of radix R over nseq sequences (stride ld) of length M.
template <int R, bool INV>
__device__ __forceinline__ void stage(const float2* __restrict__ in, float2* __restrict__ out,
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
        for (int r = 1; r < R; ++r) {
            float2 w = __ldg(&tw[k * r * tstep]);
            if (INV) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
        dft_small<R, INV>(v);
        const int base = (j / Ns) * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
    }
}

// Full transform; data starts in a, scratch b; returns the buffer holding
// the result.  Ends with a __syncthreads().
template <bool INV>
__device__ float2* fft_smem(float2* a, float2* b, const FftPlan& fp, int nseq, int ld,
                            const float2* __restrict__ tw)
{
    int Ns = 1;
    for (int s = 0; s < fp.nstages; ++s) {
        const int R = fp.radix[s];
        switch (R) {
        case 4: stage<4, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        case 2: stage<2, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        case 3: stage<3, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        default: stage<5, INV>(a, b, fp.M, Ns, nseq, ld, tw); break;
        }
        __syncthreads();
        float2* t = a;
        a = b;
        b = t;
        Ns *= R;
    }
    return a;
}

// Row transforms: rows [0, rows) of `in` (stride ld_in, first n_in entries
// nonzero) -> `out` (stride ld_out, first n_out entries kept).  With dotx,
// also Re<dotx[row][i], out[row][i]> for i < n_out, reduced per block and
// finished by the last block into scal[dot_scalar].
template <bool INV>
__global__ void k_fft_rows(const float2* in, int ld_in, int n_in, int rows, float2* out,
                           int ld_out, int n_out, FftPlan fp, const float2* __restrict__ tw,
                           int rows_per_cta, const float2* __restrict__ dotx, double* part,
                           unsigned* counter, double* scal, int dot_scalar)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    float2* a = sm;
    float2* b = sm + rows_per_cta * M;
    const int r0 = blockIdx.x * rows_per_cta;
    const int nr = min(rows_per_cta, rows - r0);
    for (int e = threadIdx.x; e < nr * M; e += blockDim.x) {
        const int q = e / M, i = e - q * M;
        a[q * M + i] = i < n_in ? in[(int64_t)(r0 + q) * ld_in + i] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_smem<INV>(a, b, fp, nr, M, tw);
    float acc = 0.f;
    for (int e = threadIdx.x; e < nr * n_out; e += blockDim.x) {
        const int q = e / n_out, i = e - q * n_out;
        const float2 v = res[q * M + i];
        const int64_t o = (int64_t)(r0 + q) * ld_out + i;
        out[o] = v;
        if (dotx) {
            const float2 xv = dotx[o];
            acc = fmaf(xv.x, v.x, fmaf(xv.y, v.y, acc));
        }
    }
    if (dotx) {
        const double tot = block_sum((double)acc);
        if (threadIdx.x == 0) part[blockIdx.x] = tot;
        if (last_block(counter)) {
            const double s = sum_parts(part, gridDim.x);
            if (threadIdx.x == 0) {
                scal[dot_scalar] = s;
                *counter = 0u;
            }
        }
    }
}

// Column pass of the Toeplitz apply: for columns [x0, x0+cpc) of the N x M
// buffer X: FFT of the N nonzero rows, multiply by Chat[x][ky], IFFT, keep
// rows < N.  Sequences sit at stride M+1 in shared memory (bank spread).
__global__ void k_fft_cols_filter(float2* X, int N, FftPlan fp, const float2* __restrict__ tw,
                                  const float* __restrict__ Chat, int cpc)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    const int ld = M + 1;
    float2* a = sm;
    float2* b = sm + cpc * ld;
    const int x0 = blockIdx.x * cpc;
    const int nc = min(cpc, M - x0);
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int y = e / nc, c = e - y * nc;
        a[c * ld + y] = y < N ? X[(int64_t)y * M + x0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2* res = fft_smem<false>(a, b, fp, nc, ld, tw);
    float2* other = res == a ? b : a;
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int c = e / M, ky = e - c * M;
        const float h = __ldg(&Chat[(int64_t)(x0 + c) * M + ky]);
        const float2 v = res[c * ld + ky];
        res[c * ld + ky] = make_float2(v.x * h, v.y * h);
    }
    __syncthreads();
    float2* res2 = fft_smem<true>(res, other, fp, nc, ld, tw);
    for (int e = threadIdx.x; e < nc * N; e += blockDim.x) {
        const int y = e / nc, c = e - y * nc;
        X[(int64_t)y * M + x0 + c] = res2[c * ld + y];
    }
}

// Column FFTs of the M x M circulant and the real spectrum:
// Chat[x][ky] = Re(FFT2 c)[ky][x] / M^2.
__global__ void k_fft_cols_spectrum(const float2* cwork, FftPlan fp, const float2* __restrict__ tw,
                                    float* Chat, int cpc)
{
    extern __shared__ float2 sm[];
    const int M = fp.M;
    const int ld = M + 1;
    float2* a = sm;
    float2* b = sm + cpc * ld;
    const int x0 = blockIdx.x * cpc;
    const int nc = min(cpc, M - x0);
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int y = e / nc, c = e - y * nc;
        a[c * ld + y] = cwork[(int64_t)y * M + x0 + c];
    }
    __syncthreads();
    float2* res = fft_smem<false>(a, b, fp, nc, ld, tw);
    const float inv = 1.0f / ((float)M * (float)M);
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int c = e / M, ky = e - c * M;
        Chat[(int64_t)(x0 + c) * M + ky] = res[c * ld + ky].x * inv;
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

constexpr int kFftSmemCap = 200 * 1024;

int rows_per_cta(int M) { return M >= 1024 ? 1 : 1024 / M; }
int cols_per_cta(int M)
{
    int c = M >= 1024 ? 4 : (M >= 512 ? 8 : 16);
    const int cap = kFftSmemCap / (2 * (M + 1) * (int)sizeof(float2));
    return c < cap ? c : (cap < 1 ? 1 : cap);
}

}  // namespace

int fft_setup_attributes(int)
{
    // one fixed ceiling for every plan: per-function attributes are global
    const int bytes = kFftSmemCap;
    SPIREC_CK(cudaFuncSetAttribute(k_fft_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_fft_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_fft_cols_filter, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    SPIREC_CK(cudaFuncSetAttribute(k_fft_cols_spectrum, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return SPIREC_OK;
}

int launch_toeplitz(spirec_plan p, const float2* x, float2* Tx, int dot_scalar)
{
    const int N = p->N, M = p->M;
    const int rpc = rows_per_cta(M);
    const int cpc = cols_per_cta(M);
    const size_t rbytes = 2 * (size_t)rpc * M * sizeof(float2);
    const size_t cbytes = 2 * (size_t)cpc * (M + 1) * sizeof(float2);
    const int threads = 256;
    const int rblocks = (N + rpc - 1) / rpc;
    k_fft_rows<false><<<rblocks, threads, rbytes, p->stream>>>(
        x, N, N, N, p->X, M, M, p->fft, p->twiddle, rpc, nullptr, nullptr, nullptr, nullptr, 0);
    SPIREC_CK(cudaGetLastError());
    k_fft_cols_filter<<<(M + cpc - 1) / cpc, threads, cbytes, p->stream>>>(p->X, N, p->fft, p->twiddle, p->Chat, cpc);
    SPIREC_CK(cudaGetLastError());
    const bool dot = dot_scalar >= 0;
    if (dot && rblocks > kMaxParts) return SPIREC_EUNSUPPORTED;
    k_fft_rows<true><<<rblocks, threads, rbytes, p->stream>>>(
        p->X, M, M, N, Tx, N, N, p->fft, p->twiddle, rpc, dot ? x : nullptr,
        dot ? p->part + (size_t)P_Q2 * kMaxParts : nullptr, dot ? p->counters + C_TOEP : nullptr,
        p->scal, dot ? dot_scalar : 0);
    SPIREC_CK(cudaGetLastError());
    p->launches += 3;
    return SPIREC_OK;
}

int launch_spectrum(spirec_plan p)
{
    const int N = p->N, M = p->M;
    const int rpc = rows_per_cta(M);
    const int cpc = cols_per_cta(M);
    const size_t rbytes = 2 * (size_t)rpc * M * sizeof(float2);
    const size_t cbytes = 2 * (size_t)cpc * (M + 1) * sizeof(float2);
    k_embed<<<4 * 152, 256, 0, p->stream>>>(p->G, N, M, p->cwork);
    SPIREC_CK(cudaGetLastError());
    k_fft_rows<false><<<(M + rpc - 1) / rpc, 256, rbytes, p->stream>>>(
        p->cwork, M, M, M, p->cwork, M, M, p->fft, p->twiddle, rpc, nullptr, nullptr, nullptr,
        nullptr, 0);
    SPIREC_CK(cudaGetLastError());
    k_fft_cols_spectrum<<<(M + cpc - 1) / cpc, 256, cbytes, p->stream>>>(p->cwork, p->fft, p->twiddle, p->Chat, cpc);
    SPIREC_CK(cudaGetLastError());
    p->launches += 3;
    return SPIREC_OK;
}

}  // namespace spirec
