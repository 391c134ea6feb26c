// nudft_simt.cu -- FP32 CUDA-core contractions of the exact NUDFT:
//   G (Eq. AnnMatG), D = H^H s (Eq. AnnMatGD) and y = H x (Eq. ModDirect).
//
// G and D are both "phase GEMMs": C[i][c] = scale * sum_l A(l,i) B(l,c) with
//   A(l,i) = exp(sa i2pi ka_l (i + oa)),   B(l,c) = w_l exp(sb i2pi kb_l (c + ob)),
// a complex GEMM of K = L whose operands are generated in shared memory from
// the fixed-point trajectory (phase.cuh) and never stored in HBM.  Because the
// output is small (N x (2N-1) at most) and K is huge, the sample axis is split
// over grid.z (split-K); each split writes FP32 partials and a second kernel
// sums them in a fixed order, so results do not depend on scheduling.
#include <stdint.h>

#include "internal.cuh"
#include "phase.cuh"

namespace spirec {

namespace {

constexpr int TM = 64;   // tile rows (i)
constexpr int TN = 64;   // tile cols (c)
constexpr int KC = 32;   // samples per shared-memory stage
constexpr int NT = 256;  // threads

// Generated operand tiles.  A tile entry (l, i) is base[l][i/8] * off[l][i%8]
// with base = exp(i2pi k (i0 + 8a + o)) and off = exp(i2pi k b): 16 trig calls
// per sample and tile side instead of 64.
template <bool WEIGHTED>
__global__ void __launch_bounds__(NT, 2)
k_phase_gemm(const int64_t* __restrict__ ka, const int64_t* __restrict__ kb,
             const float2* __restrict__ w, int64_t L, int R, int C, int oa, int ob, int sa,
             int sb, int64_t chunks_per_split, float2* __restrict__ part)
{
    __shared__ float2 As[KC][TM];
    __shared__ float2 Bs[KC][TN];
    __shared__ float2 tab[4][KC][8];  // baseA, offA, baseB, offB

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int i0 = blockIdx.y * TM, c0 = blockIdx.x * TN;
    const int64_t nchunks = (L + KC - 1) / KC;
    const int64_t ch0 = (int64_t)blockIdx.z * chunks_per_split;
    int64_t ch1 = ch0 + chunks_per_split;
    if (ch1 > nchunks) ch1 = nchunks;

    float2 acc[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);

    for (int64_t ch = ch0; ch < ch1; ++ch) {
        const int64_t lbase = ch * KC;
        // 1) factor tables: 4 tables x KC samples x 8 = 1024 entries
#pragma unroll
        for (int e = tid; e < 4 * KC * 8; e += NT) {
            const int t = e / (KC * 8), l = (e / 8) % KC, q = e % 8;
            const int64_t lg = lbase + l;
            float2 v = make_float2(0.f, 0.f);
            if (lg < L) {
                const bool isA = t < 2;
                const bool isBase = (t & 1) == 0;
                const int64_t k = isA ? ka[lg] : kb[lg];
                const int j = isBase ? (isA ? i0 + 8 * q + oa : c0 + 8 * q + ob) : q;
                v = phasor_q(k, j);
                if ((isA ? sa : sb) < 0) v.y = -v.y;
                if (WEIGHTED && !isA && isBase) v = cmul(v, w[lg]);
            }
            tab[t][l][q] = v;
        }
        __syncthreads();
        // 2) operand tiles
#pragma unroll
        for (int e = tid; e < KC * TM; e += NT) {
            const int l = e / TM, i = e % TM;
            As[l][i] = cmul(tab[0][l][i >> 3], tab[1][l][i & 7]);
            Bs[l][i] = cmul(tab[2][l][i >> 3], tab[3][l][i & 7]);
        }
        __syncthreads();
        // 3) complex multiply-accumulate, 4 x 4 outputs per thread
#pragma unroll 4
        for (int l = 0; l < KC; ++l) {
            float2 a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = As[l][ty + 16 * r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = Bs[l][tx + 16 * c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    acc[r][c].x = fmaf(a[r].x, b[c].x, acc[r][c].x);
                    acc[r][c].x = fmaf(-a[r].y, b[c].y, acc[r][c].x);
                    acc[r][c].y = fmaf(a[r].x, b[c].y, acc[r][c].y);
                    acc[r][c].y = fmaf(a[r].y, b[c].x, acc[r][c].y);
                }
        }
        __syncthreads();
    }
    float2* out = part + (int64_t)blockIdx.z * R * C;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int i = i0 + ty + 16 * r;
        if (i >= R) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int cc = c0 + tx + 16 * c;
            if (cc < C) out[(int64_t)i * C + cc] = acc[r][c];
        }
    }
}

// out[i*C + c] = scale * sum_s part[s][i][c], fixed summation order.
__global__ void k_reduce_splits(const float2* __restrict__ part, int S, int64_t RC, float scale,
                                float2* __restrict__ out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < RC;
         e += (int64_t)gridDim.x * blockDim.x) {
        float2 a = make_float2(0.f, 0.f);
        for (int s = 0; s < S; ++s) {
            const float2 v = part[(int64_t)s * RC + e];
            a.x += v.x;
            a.y += v.y;
        }
        out[e] = make_float2(a.x * scale, a.y * scale);
    }
}

// y = H x.  Z[n][l] = sum_m x[n][m] exp(i2pi kx_l m) as a GEMM (A = image rows,
// B = generated phases), then y_l += sum_n exp(i2pi ky_l n) Z[n][l] in the
// epilogue; the N x L intermediate never leaves registers.  grid.y splits the
// row blocks; partials ypart[split][l].
__global__ void __launch_bounds__(NT, 2)
k_forward(const int64_t* __restrict__ kxq, const int64_t* __restrict__ kyq,
          const float2* __restrict__ x, int N, int64_t L, float2* __restrict__ ypart)
{
    __shared__ float2 As[TM][KC + 1];   // image tile [row][m]
    __shared__ float2 Bs[KC][TN];       // phases [m][l]
    __shared__ float2 off[TN][8];       // exp(i2pi kx_l b), b < 8
    __shared__ float2 base[TN][KC / 8]; // exp(i2pi kx_l (m0 + 8a))
    __shared__ float2 red[16][TN];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t l0 = (int64_t)blockIdx.x * TN;
    const int nblocks = (N + TM - 1) / TM;

    for (int e = tid; e < TN * 8; e += NT) {
        const int c = e / 8, b = e % 8;
        const int64_t lg = l0 + c;
        off[c][b] = lg < L ? phasor_q(kxq[lg], b) : make_float2(0.f, 0.f);
    }
    float2 yacc = make_float2(0.f, 0.f);  // thread c < TN owns sample l0 + c

    for (int nb = blockIdx.y; nb < nblocks; nb += gridDim.y) {
        const int n0 = nb * TM;
        float2 acc[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = make_float2(0.f, 0.f);

        for (int m0 = 0; m0 < N; m0 += KC) {
            __syncthreads();
            for (int e = tid; e < TN * (KC / 8); e += NT) {
                const int c = e / (KC / 8), a = e % (KC / 8);
                const int64_t lg = l0 + c;
                base[c][a] = lg < L ? phasor_q(kxq[lg], m0 + 8 * a) : make_float2(0.f, 0.f);
            }
            for (int e = tid; e < TM * KC; e += NT) {
                const int r = e / KC, k = e % KC;
                const int n = n0 + r, m = m0 + k;
                As[r][k] = (n < N && m < N) ? x[(int64_t)n * N + m] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            for (int e = tid; e < KC * TN; e += NT) {
                const int k = e / TN, c = e % TN;
                Bs[k][c] = cmul(base[c][k >> 3], off[c][k & 7]);
            }
            __syncthreads();
#pragma unroll 4
            for (int k = 0; k < KC; ++k) {
                float2 a[4], b[4];
#pragma unroll
                for (int r = 0; r < 4; ++r) a[r] = As[ty + 16 * r][k];
#pragma unroll
                for (int c = 0; c < 4; ++c) b[c] = Bs[k][tx + 16 * c];
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        acc[r][c].x = fmaf(a[r].x, b[c].x, acc[r][c].x);
                        acc[r][c].x = fmaf(-a[r].y, b[c].y, acc[r][c].x);
                        acc[r][c].y = fmaf(a[r].x, b[c].y, acc[r][c].y);
                        acc[r][c].y = fmaf(a[r].y, b[c].x, acc[r][c].y);
                    }
            }
        }
        // epilogue: sum_n exp(i2pi ky_l n) Z[n][l] over this row block
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t lg = l0 + tx + 16 * c;
            float2 sacc = make_float2(0.f, 0.f);
            if (lg < L) {
                const int64_t k = kyq[lg];
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int n = n0 + ty + 16 * r;
                    if (n < N) {
                        const float2 e = cmul(phasor_q(k, n), acc[r][c]);
                        sacc.x += e.x;
                        sacc.y += e.y;
                    }
                }
            }
            red[ty][tx + 16 * c] = sacc;
        }
        __syncthreads();
        if (tid < TN) {
            for (int r = 0; r < 16; ++r) {
                yacc.x += red[r][tid].x;
                yacc.y += red[r][tid].y;
            }
        }
    }
    if (tid < TN && l0 + tid < L) ypart[(int64_t)blockIdx.y * L + l0 + tid] = yacc;
}

// Sample slices of the contraction: the tuned value of the shape, else about
// six resident CTAs per SM over the device; bounded by the work and by the
// partial-sum buffer.
int choose_splits(spirec_plan p, int knob, int sms, int64_t tiles, int64_t nchunks, int64_t RC)
{
    const size_t part_cap_elems = p->kpart_bytes / sizeof(float2);
    const int tuned = tune_lookup(knob, p, sms);
    int64_t S = tuned > 0 ? tuned : (6 * sms + tiles - 1) / tiles;
    if (S > nchunks) S = nchunks;
    if (S < 1) S = 1;
    while (S > 1 && (size_t)(S * RC) > part_cap_elems) --S;
    return (int)S;
}

void simt_shape(const spirec_plan_s* p, int knob, int* R, int* C)
{
    *R = p->N;
    *C = knob == SPIREC_KNOB_GRAM_SPLIT ? 2 * p->N - 1 : p->N;
}

int phase_gemm(spirec_plan p, int knob, const int64_t* ka, const int64_t* kb, const float2* w, int R,
               int C, int oa, int ob, int sa, int sb, float scale, float2* out)
{
    const int64_t nchunks = (p->L + KC - 1) / KC;
    const int64_t tiles = (int64_t)((R + TM - 1) / TM) * ((C + TN - 1) / TN);
    const int64_t RC = (int64_t)R * C;
    int sms = 0, rc;
    if ((rc = device_sms(&sms)) != SPIREC_OK) return rc;
    const int S = choose_splits(p, knob, sms, tiles, nchunks, RC);
    const int64_t cps = (nchunks + S - 1) / S;
    const int Seff = (int)((nchunks + cps - 1) / cps);
    dim3 grid((C + TN - 1) / TN, (R + TM - 1) / TM, Seff);
    float2* part = reinterpret_cast<float2*>(p->kpart);
    if (w)
        k_phase_gemm<true><<<grid, NT, 0, p->stream>>>(ka, kb, w, p->L, R, C, oa, ob, sa, sb, cps, part);
    else
        k_phase_gemm<false><<<grid, NT, 0, p->stream>>>(ka, kb, w, p->L, R, C, oa, ob, sa, sb, cps, part);
    SPIREC_CK(cudaGetLastError());
    int rblocks = (int)((RC + 255) / 256);
    if (rblocks > 4 * 152) rblocks = 4 * 152;
    k_reduce_splits<<<rblocks, 256, 0, p->stream>>>(part, Seff, RC, scale, out);
    SPIREC_CK(cudaGetLastError());
    p->launches += 2;
    return SPIREC_OK;
}

}  // namespace

int launch_gram(spirec_plan p)
{
    if (p->precision != SPIREC_FP32) return launch_gram_tc(p);
    const int N = p->N;
    // G[u][v+N-1] = (1/N^2) sum_l exp(i2pi kx_l u) exp(i2pi ky_l v)
    return phase_gemm(p, SPIREC_KNOB_GRAM_SPLIT, p->kxq, p->kyq, nullptr, N, 2 * N - 1, 0, -(N - 1), +1, +1,
                      1.0f / ((float)N * (float)N), p->G);
}

int launch_adjoint(spirec_plan p, const float2* y, float2* x)
{
    if (p->precision != SPIREC_FP32) return launch_adjoint_tc(p, y, x);
    const int N = p->N;
    // x[n][m] = (1/N) sum_l exp(-i2pi ky_l n) * (y_l exp(-i2pi kx_l m))
    return phase_gemm(p, SPIREC_KNOB_ADJOINT_SPLIT, p->kyq, p->kxq, y, N, N, 0, 0, -1, -1, 1.0f / (float)N, x);
}

int contraction_split(spirec_plan p, int knob, int* value, int* sms_used)
{
    int sms = 0, rc;
    if ((rc = device_sms(&sms)) != SPIREC_OK) return rc;
    if (p->precision != SPIREC_FP32) {
        int64_t P = 0;
        if ((rc = tc_ctas(p, knob, sms, &P)) != SPIREC_OK) return rc;
        *value = (int)P;
        *sms_used = (int)P;  // one CTA per SM (its shared memory)
        return SPIREC_OK;
    }
    int R = 0, C = 0;
    simt_shape(p, knob, &R, &C);
    const int64_t nchunks = (p->L + KC - 1) / KC;
    const int64_t tiles = (int64_t)((R + TM - 1) / TM) * ((C + TN - 1) / TN);
    const int S = choose_splits(p, knob, sms, tiles, nchunks, (int64_t)R * C);
    const int64_t cps = (nchunks + S - 1) / S;
    const int64_t blocks = tiles * ((nchunks + cps - 1) / cps);
    int per_sm = 0;
    SPIREC_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_phase_gemm<true>, NT, 0));
    if (per_sm < 1) per_sm = 1;
    const int64_t used = (blocks + per_sm - 1) / per_sm;
    *value = S;
    *sms_used = (int)(used < sms ? used : sms);
    return SPIREC_OK;
}

int launch_forward(spirec_plan p, const float2* x, float2* y)
{
    if (p->precision != SPIREC_FP32) return launch_forward_tc(p, x, y);
    const int64_t lblocks = (p->L + TN - 1) / TN;
    const int nblocks = (p->N + TM - 1) / TM;
    int ns = (int)((4 * 152 + lblocks - 1) / lblocks);
    if (ns > nblocks) ns = nblocks;
    if (ns < 1) ns = 1;
    while (ns > 1 && (size_t)ns * p->L * sizeof(float2) > p->kpart_bytes) --ns;
    float2* part = reinterpret_cast<float2*>(p->kpart);
    dim3 grid((unsigned)lblocks, ns);
    k_forward<<<grid, NT, 0, p->stream>>>(p->kxq, p->kyq, x, p->N, p->L, part);
    SPIREC_CK(cudaGetLastError());
    int rblocks = (int)((p->L + 255) / 256);
    if (rblocks > 4 * 152) rblocks = 4 * 152;
    k_reduce_splits<<<rblocks, 256, 0, p->stream>>>(part, ns, p->L, 1.0f / (float)p->N, y);
    SPIREC_CK(cudaGetLastError());
    p->launches += 2;
    return SPIREC_OK;
}

}  // namespace spirec
