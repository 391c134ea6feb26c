// internal.cuh -- shared declarations of the CUDA path (plan state, device
// helpers, kernel launchers).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/spirec.h"
#include "penalty.cuh"

namespace spirec {

// ------------------------------------------------------------ error helpers

void set_error(const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* what);

#define SPIREC_CK(call)                                        \
    do {                                                       \
        cudaError_t e__ = (call);                              \
        if (e__ != cudaSuccess) return cuda_fail(e__, #call);  \
    } while (0)

// ---------------------------------------------------------------- FFT plan

constexpr int kMaxStages = 16;
struct FftPlan {
    int M;
    int nstages;
    int radix[kMaxStages];
};
bool make_fft_plan(int M, FftPlan* p);

// ----------------------------------------------------------- partial sums

// Slots of the block-partial array (float-float pairs, kMaxParts per slot,
// one per block of the kernel that produced them).
constexpr int kMaxParts = 4096;
enum PartSlot {
    P_ROWA = 0,   // row pass 1 of the CG: q1, num0, den0 (3 slots)
    P_ROWC = 3,   // row pass 3: q2 (or a plain dot)
    P_LS = 4,     // line-search step: num, den (2 slots)
    P_UPD = 6,    // gradient/update: 6 slots (see k_update)
    P_MISC = 12,  // one-off sums (2 slots)
    P_NSLOTS = 14
};
constexpr int kUpdVals = 6;  // sums of the update kernel

// Arrival counters of the last-block reductions, one per kernel kind.
enum Counter {
    C_ROWA = 0, C_ROWC = 1, C_LS = 2, C_UPD = 3, C_MISC = 4, C_AMAX = 5,
    C_BAR = 8,  // grid barrier of the persistent loop: arrivals, generation, abort
    C_N = 16
};

// Bits of the device error word (plan->dflag).
enum DeviceError { E_TRAJ = 1, E_TIMEOUT = 2 };

// Device scalars (FP64), written by the last block of the kernel that
// reduces them and read by later kernels in stream order.
enum Scalar {
    S_SS = 0,     // ||s||^2
    S_Q1 = 1,     // Re<d, g_ls>
    S_Q2 = 2,     // ||H d||^2 = Re<d, T d>
    S_T1 = 3,     // line-search steps t1, t2, t3 (S_T1 + j)
    S_T3 = 5,
    S_GG = 6,     // <g, g> of the current gradient
    S_BETA = 7,   // Polak-Ribiere beta for the next direction (0 = restart)
    S_J = 8,      // J of the current iterate
    S_R = 9,      // R of the current iterate
    S_TMP = 10,   // result of a one-off dot
    S_NUM0 = 11,  // penalty part of h'(0)
    S_DEN0 = 12,  // penalty part of the majorant curvature at t = 0
    S_HQ_RHO = 13,    // half-quadratic inner CG: <r, r>
    S_HQ_ALPHA = 14,  //   step alpha
    S_HQ_BETA = 15,   //   direction beta
    S_PROF = 16,  // 16 slots: time (ns) block 0 of the persistent loop spent per phase
    S_NSCAL = 32
};

struct Reg {
    float lambda1, alpha1, lambda0, alpha0;
    int kind;
};

// Pointers of the fused CG passes (row pass 1 and 3 of the Toeplitz apply).
struct CgPass {
    const float2* g;
    const float2* d_old;
    float2* d_new;
    const float2* f;
    const float2* res;  // T f - D, the data term's image-domain residual
    const float2* D;
    Reg reg;
    float2* parts;
    unsigned* counter;
    double* scal;
};

// ------------------------------------------------------------------- plan

}  // namespace spirec

struct spirec_plan_s {
    int N;
    int64_t L;
    int M;
    int precision;
    int device;
    cudaStream_t user_stream;
    cudaStream_t stream;  // own, non-blocking
    cudaEvent_t ev_join;
    // host data upload beside the plan's stream (spirec_set_data): the
    // caller's s goes to s_in on copy_stream, then the plan's stream moves it
    // into s; made on first use
    cudaStream_t copy_stream;
    cudaEvent_t ev_s_ready;   // s_in holds the caller's data
    cudaEvent_t ev_sin_free;  // the plan's stream has moved s_in into s
    cudaEvent_t ev_traj_in;   // a host trajectory is on the device (spirec_set_trajectory)
    float2* s_in;             // L (+32)

    // trajectory, fixed point: k * 2^64 mod 2^64
    int64_t* kxq;
    int64_t* kyq;
    // the weights of a paired tensor-core contraction (mixed precisions; 32
    // zero entries of padding): w_l times the phase of the pairing's centre
    float2* wpair;
    double* kstage;  // 2L: host trajectory staged on the device
    int* dflag;  // device error flag
    // two pinned host words, made on first use: the last J of a host solve
    // and (as an int) a copy of dflag, so that a host call's copies all go
    // asynchronously and it synchronises once
    double* hpin;

    float2* G;     // N x (2N-1)
    float* Chat;   // M x M real, transposed: Chat[kx*M + ky]
    float2* cwork; // M x M complex (spectrum build)
    float2* X;     // N x M complex (Toeplitz rows)
    float2* D;     // N x N
    float2* s;     // L (+32 padding)
    float2* ystage;  // L (+32 padding): a caller's y staged for the tensor-core adjoint
    float2* f[2];
    float2* dbuf[2];  // direction of iteration k in dbuf[k & 1]
    float2* g;
    float2* res;   // T f - D of the iterate (the data term's gradient is 2 res)
    float2* Td;
    float2* tmp;   // N x N scratch for operator calls
    float2* twiddle;  // M entries, exp(-2 pi i k / M)
    double* part;  // P_NSLOTS x kMaxParts (float-float pairs)
    double* scal;  // S_NSCAL
    unsigned* counters;  // C_N
    double* Jdev;  // J history (device), capacity Jcap
    int Jcap;
    uint8_t* fsplit;  // the image split into hi/lo operand tiles (tensor-core forward)
    size_t fsplit_bytes;
    float* kpart;  // split-K partial sums of the contractions
    size_t kpart_bytes;
    size_t device_bytes;

    spirec::FftPlan fft;
    spirec::Reg reg;
    bool have_traj, have_data, have_reg;

    // kernels launched (graph replays count every kernel node)
    int64_t launches;
    int64_t graph_kernels;

    // CUDA graph of the iteration loop
    cudaGraphExec_t graph;
    int graph_iters;
    unsigned graph_tune_gen;  // tuning-table generation the graph was captured under
    int graph_parity_out;
    int result_slot;  // the last solve left its iterate in f[result_slot]
    int mode;         // SPIREC_MODE_TOEPLITZ or SPIREC_MODE_DIRECT
    int minimiser;    // SPIREC_MIN_PRCG, SPIREC_MIN_HALF_QUADRATIC or SPIREC_MIN_NEWTON
    int hq_inner;     // linear CG steps per half-quadratic or Newton outer step
    float* hqw;       // 6 x N x N weights W, then E (right edge, down edge, pixel each)
    float2* ydir;     // L (+32): H d of the direct mode

    // timing
    bool timing;
    cudaEvent_t tev[2 * 64];
    bool tev_made[2 * 64];
    int tev_stage[64];
    int tev_used;
    double t_ms[SPIREC_NUM_STAGES];
    int64_t t_cnt[SPIREC_NUM_STAGES];
};

namespace spirec {

// -------------------------------------------------------------- launchers
// All launchers enqueue on p->stream and return a spirec_status.

int launch_gram(spirec_plan p);            // G from the trajectory
int launch_spectrum(spirec_plan p);        // Chat from G
int launch_adjoint(spirec_plan p, const float2* y, float2* x);  // x = H^H y
int launch_forward(spirec_plan p, const float2* x, float2* y);  // y = H x

// Toeplitz T x -> Tx; with dot_scalar >= 0 also scal[dot_scalar] = Re<x, Tx>.
int launch_toeplitz(spirec_plan p, const float2* x, float2* Tx, int dot_scalar);
int fft_setup_attributes(int maxM);
// Toeplitz passes; mode 1 = the fused CG forms (see fft.cu).
int launch_rows_fwd(spirec_plan p, const float2* in, int ld_in, int n_in, int rows, int mode,
                    const CgPass* cg);
int launch_cols(spirec_plan p, int n_in, int n_out);
int launch_rows_inv(spirec_plan p, float2* out, int mode, const float2* dotx, const CgPass* cg,
                    int dot_scalar);

// CG pieces (cg.cu).  Iteration k reads f[k & 1] and writes f[(k + 1) & 1].
int launch_data_norm(spirec_plan p);
// res = Tx - D where res holds T x (have_tx), else res = -D (x = 0)
int launch_res_init(spirec_plan p, float2* res, bool have_tx);
// gradient at f (res = T f - D given): g, J -> Jout, <g,g>; first = no step taken
int launch_update(spirec_plan p, const float2* f_in, float2* f_out, const float2* d, float2* res,
                  const float2* Td, float2* g, int first, double* Jout);
int launch_line_search(spirec_plan p, const float2* f, const float2* d, int step);
int cg_iteration(spirec_plan p, int k, double* Jdev);
// T x as H^H (H x) (direct mode); with dot_q2_t1 also q2 = Re<x, T x> and the
// first line-search step into scal (as the fused row pass of the FFT path).
int launch_normal_direct(spirec_plan p, const float2* x, float2* Tx, bool dot_q2_t1);
// Half-quadratic minimiser (halfquad.cu): J of f[0] (and the weights at it)
// into Jout; one outer step k (weights, J(f^k) -> Jdev[k], hq_inner linear
// CG steps on the frozen quadratic), iterate in f[0].
int launch_hq_objective(spirec_plan p, double* Jout);
int hq_outer_step(spirec_plan p, int k, double* Jdev);
// Truncated Newton minimiser (halfquad.cu): one outer step k (J(f^k) ->
// Jdev[k], hq_inner CG steps on the Newton system, the line search, the step).
int nt_outer_step(spirec_plan p, int k, double* Jdev);
// The whole loop (first gradient + iters iterations) as one persistent
// cooperative kernel (cg_loop.cu); power-of-two M in [64, 2048] only, and
// SPIREC_EUNSUPPORTED (nothing enqueued) when the image does not fit its
// shared-memory caches.  The iterate ends in f[0].
bool loop_supported(int M);
int launch_cg_loop(spirec_plan p, int iters);

// tensor-core contractions (FP16x3 / BF16x3)
int launch_gram_tc(spirec_plan p);
int launch_adjoint_tc(spirec_plan p, const float2* y, float2* x);
int launch_forward_tc(spirec_plan p, const float2* x, float2* y);
size_t fsplit_bytes_tc(int N, int precision);  // the forward's split-image buffer
size_t kpart_floats_tc(int N, int64_t L, int precision);  // split-K buffer need
int tc_setup_attributes();

// Tuned launch parameters (tune.cu).  tune_lookup gives the table entry of
// the plan's shape for the knob on a device with `sms` SMs, 0 if none;
// tune_store sets (value > 0) or removes it.  The generation grows with every
// change (graphs captured under an older one are re-captured).
int l_class(int64_t L);
int tune_lookup(int knob, const spirec_plan_s* p, int sms);
int tune_store(int knob, const spirec_plan_s* p, int sms, int value);
unsigned tune_generation();
int device_sms(int* sms);

// The split of the G (SPIREC_KNOB_GRAM_SPLIT) or D (SPIREC_KNOB_ADJOINT_SPLIT)
// contraction that a launch of this plan uses now (the table entry, else the
// heuristic, clipped), and the SMs it occupies (nudft_simt.cu).
int contraction_split(spirec_plan p, int knob, int* value, int* sms_used);
// Loop shapes the plan can launch: rows per block and grid, at most `max`
// (cg_loop.cu); the shape a launch uses now.
int loop_candidates(spirec_plan p, int* RB, int* grid, int max);
int loop_current(spirec_plan p, int* RB, int* grid);
// Blocks the persistent loop of the plan's current shape launches, and how
// many blocks of that shape the device holds at once (1 when it has a shape;
// 0 and nothing set otherwise).  A cooperative launch needs all its blocks
// resident together, so concurrent loops must fit that capacity jointly.
int loop_demand(spirec_plan p, int* blocks, int* capacity);
// The same for the plan's next solve: 0 blocks when it will not run the
// persistent loop (direct mode, another minimiser, M without a loop).
int solve_loop_demand(spirec_plan p, int* blocks, int* capacity);
// Device bytes the request loop reserves for a request of this shape, and the
// grid side M it plans it with (server.cu).
size_t server_plan_bytes(int N, int64_t L, int precision, int* M);
int tc_ctas(spirec_plan p, int knob, int sms, int64_t* P);  // nudft_tc.cu
// The tile shape the contraction of a split knob uses now: CTA pairs (true)
// or one SM a tile (nudft_tc.cu).
bool tc_pairs(spirec_plan p, int knob, int sms);

// Limit of every bounded device wait of the kernels launched from now on
// (2 s unless spirec_set_wait_limit_ns changed it).
unsigned long long wait_limit_ns();
// Kernels a test has asked to stall (spirec_inject_wait_stall): such a launch
// waits once on a condition nothing fulfils, so its bounded wait runs out.
constexpr int kStallLoop = 1;         // the persistent CG loop
constexpr int kStallContraction = 2;  // the tensor-core contractions
bool injected_stall(int kind);

int vec_blocks(int N);
constexpr int kVecThreads = 256;
constexpr int kVecBlocksPerSm = 5;  // resident blocks an SM the vector kernels are built for

}  // namespace spirec
