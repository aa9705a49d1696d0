// Internal declarations shared by the host plan code and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "sfrd.h"

namespace sfrd {

constexpr int kMaxStages = 16;
constexpr int kMaxFFT = 1024;   // longest complex FFT along one axis
constexpr int kThreads = 256;   // threads per block of every transform pass

// Per-axis description handed to kernels by value.
struct AxisDev {
    int n;        // unknowns along the axis
    int N;        // intervals
    int M;        // complex FFT length: N (periodic) or 2N (Dirichlet/Neumann extension)
    int bc;       // SFRD_BC_*
    int nst;      // radix stages
    int radix[kMaxStages];   // DIF order; DIT runs them reversed
    const void* tw;          // omega_M^k = exp(-2 pi i k / M), k < M, in the run precision
    const int* perm;         // extension index -> buffer slot after DIF (= DIT input slot)
    int node0;               // grid node of unknown 0 (1 for Dirichlet, else 0)
    double lo, h;            // node coordinate = lo + (node0 + i) h
};

struct ReactDev {
    int kind;
    int S;
    double p[8];
    double off[2];
    double c[2];   // Schnakenberg: (a - u0 + u0^2 v0, b - u0^2 v0) at the offset (u0, v0), in FP64
};

// Device-resident clock: t_k = t0 + k tau (Algorithm 1).
struct Clock {
    double t0;
    long long k;
};

// Transform pass kinds.
enum PassMode {
    MODE_PLAIN = 0,  // one transform along the axis, out = scale * T(in)
    MODE_T0 = 1,     // slow axis: F = T(in); U <- F; out = T(U)/C
    MODE_TA = 2,     // slow axis: F1 <- T(in); out = T(Q U + phi F1)/C
    MODE_TB = 3,     // slow axis: F2 <- T(in); out = T(Q U + phi F2)/C
    MODE_TC = 4,     // slow axis: F3 <- T(in); out = T(Q(Q U + phi F1) + phi(2F3 - F1))/C
    MODE_TD = 5,     // slow axis: U <- R U + phi1 F1 + phi2 (F2+F3) + phi3 T(in); out = T(U)/C
    MODE_REACT = 6,  // contiguous axis: out = T(f(T(in)))
    // discrete adjoint (register engine only; tilde-frame cotangents, see adjoint.cuh)
    MODE_XADJ = 7,       // contiguous axis: out = T(J_f(state)^T T(in)); accumulates dL/dparams
    MODE_ADJ_ENTRY = 8,  // slow axis: out = T(phi3 Ub)
    MODE_ADJ_CB = 9,     // slow axis: Cb = T(in)/C; out = T(phi2 Ub + 2 phi Cb)
    MODE_ADJ_BA = 10,    // slow axis: Bb = T(in)/C; out = T(phi2 Ub + phi Bb)
    MODE_ADJ_AU = 11,    // slow axis: Ab = Q Cb + T(in)/C; out = T(phi1 Ub - phi Cb + phi Ab)
    MODE_ADJ_EXIT = 12,  // slow axis: Ub <- R Ub + Q Bb + Q Ab + T(in)/C
};

// Pass kinds reported by the per-launch profile of one step.
enum PassKind { PASS_X = 0, PASS_MID = 1, PASS_SLOW_A = 2, PASS_SLOW_B = 3, PASS_SLOW_C = 4, PASS_SLOW_D = 5 };

template <typename T>
struct ColArgs {
    const T* in;
    T* out;
    long long in_offB;    // element offset from real column A to real column B
    long long in_sAxis;   // stride along the transformed axis
    long long in_sOther;  // stride of the blockIdx.y coordinate
    long long out_offB, out_sAxis, out_sOther;   // same for the output array
    int in_xlim;          // columns x < in_xlim are loaded (others read as 0)
    int out_xlim;         // columns x < out_xlim are stored
    int xw;               // x advance per blockIdx.x
    int bshift;           // column of line B minus column of line A (0: other species; CC: same species)
    double scale;         // output scale (plain mode)
    double invC;          // 1/C for the slow-axis inverse (T modes)
    T* U;
    T* F1;
    T* F2;
    T* F3;
    const T* CQ;          // interleaved (Q13, phi) pairs
    const T* CR;          // interleaved (R13, phi1, phi2, phi3) quads
    Clock* clock;         // TD advances k
    AxisDev ax;
    T* F4;                // MODE_TD: F(f_c) of the step is also stored here when non-null
    // adjoint
    T* Ub;                // spectral cotangent of the state (tilde frame), read; updated by ADJ_EXIT
    T* Cb;
    T* Bb;
    T* Ab;
    double* grad;         // [0,1] dL/dkappa_s, [2,3] dL/dalpha_s (atomic accumulation)
    const double* lam[3]; // eigenvalue tables (x, y, z)
    int nk[3];            // unknowns per axis (x, y, z)
    int dim;
    int S;
    double alpha[2], kappa[2], tau;
    int scheme;           // SFRD_SCHEME_*: which coefficients the adjoint differentiates
    // SFRD_COEF_RATIONAL: the slow-axis combinations evaluate the coefficients from L = cl_mult[h] *
    // CL[i + (h ? clB : 0)] (line h of the tile); CL == nullptr with stored coefficient arrays.  On the
    // element-pair grid (species s = blockIdx.z, both lines of species s) the L of element i of species
    // s is cl_mult[s] * CL[i - s * (in_sp - cl_sp)]: cl_sp is the species stride of CL (0 when the
    // species share one plane of tau Lambda^{alpha/2}).
    const T* CL;
    double cl_mult[2];
    long long clB, cl_sp;
    int cstride;          // x distance between the tile columns of neighbouring lanes (2: lines A and B
                          // are the adjacent columns x, x + 1 of one array, read and written as pairs)
    long long in_sp, out_sp;   // species stride (elements) of blockIdx.z; 0 when species are tile lines
};

template <typename T>
struct XArgs {
    const T* in;
    T* out;
    long long in_offB, out_offB;      // element offset from row A to row B
    long long in_pitch, out_pitch;    // row strides
    int rows;                         // (z, y) rows per species
    int out_fill;                     // zero-fill columns n..out_fill-1 of each output row
    int S;
    int ny;                           // rows -> (y, z) for coordinates
    double tau, stage_frac;           // reaction time = t0 + (k + stage_frac) tau
    const Clock* clock;
    AxisDev ax, ay, az;
    ReactDev re;
    T* save;              // MODE_REACT: physical stage values also stored here when non-null
    const T* state;       // MODE_XADJ: stored physical stage values (same layout as in/out)
    double* grad;         // MODE_XADJ: dL/dparams accumulators [8]
    int nz;
};

// Host-side plan.
struct Plan {
    int dim = 0, bc = 0, dtype = 0, S = 0;
    int64_t Nint[3] = {1, 1, 1};
    double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
    int n[3] = {1, 1, 1};      // unknowns (x, y, z)
    int M[3] = {1, 1, 1};
    int pitch = 0;             // internal row pitch (elements), multiple of 4
    long long plane = 0;       // internal elements per species: n_z * n_y * pitch
    long long dense = 0;       // dense elements per species: n_z * n_y * n_x
    double alpha[2] = {0, 0}, kappa[2] = {0, 0};
    double dt = 0;
    ReactDev re{};
    int CC = 16;               // complex columns per tile (generic engine)
    bool v2[3] = {false, false, false};   // axis uses the register FFT engine
    size_t esize = 8;

    // host tables (kept alive for async uploads)
    std::vector<double> lam[3];
    std::vector<double> tw64[3];   // interleaved re, im
    std::vector<float> tw32[3];
    std::vector<int> perm[3];
    std::vector<int> radix[3];

    // workspace layout (byte offsets)
    size_t off_W = 0, off_W2 = 0, off_U = 0, off_F1 = 0, off_F2 = 0, off_F3 = 0;
    size_t off_CQ = 0, off_CR = 0, off_clock = 0, off_D = 0;
    int coef_mode = 0;          // SFRD_COEF_STORED or SFRD_COEF_RATIONAL
    bool cl_shared = false;     // rational mode: one plane tau Lambda^{alpha/2} for both species
    int sched_rule = 0;         // radix-order rule of the shared-memory engine (apply_schedule)
    int scheme = 0;             // SFRD_SCHEME_P13 or SFRD_SCHEME_COX_MATTHEWS
    bool debug_checks = false;  // SFRD_DEBUG_CHECKS set at plan creation: check the state after advance
    size_t off_flag = 0;        // device int written by the non-finite check
    size_t off_CL = 0;
    size_t off_tw[3] = {0, 0, 0}, off_perm[3] = {0, 0, 0}, off_lam[3] = {0, 0, 0};
    size_t ws_bytes = 0;

    char* ws = nullptr;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    cudaGraph_t step_graph = nullptr;
    bool loaded = false;
};

// Launchers (sfrd_passes_*.cu), templated on the run precision.
template <typename T> cudaError_t launch_step(Plan& p, cudaStream_t s);
template <typename T> cudaError_t launch_step_profiled(Plan& p, cudaStream_t s, cudaEvent_t* ev, int* kind, int cap);
template <typename T> cudaError_t launch_load(Plan& p, const void* u0, cudaStream_t s);
template <typename T> cudaError_t launch_store(Plan& p, void* u, cudaStream_t s);
template <typename T> cudaError_t launch_forward(Plan& p, const void* u, void* uhat, cudaStream_t s);
template <typename T> cudaError_t launch_inverse(Plan& p, const void* uhat, void* u, cudaStream_t s);
template <typename T> cudaError_t launch_coef_init(Plan& p, cudaStream_t s);
template <typename T> cudaError_t launch_finite_check(Plan& p, cudaStream_t s);
template <typename T> cudaError_t launch_coef_copy(Plan& p, int which, void* out, cudaStream_t s);
template <typename T> cudaError_t prepare_kernels(const Plan& p);

// Register-FFT passes for power-of-two axis lengths (passes2.cuh, one translation unit per length).
namespace v2 {
constexpr int kMaxDynSmem2 = 227 * 1024;
constexpr int kMinN = 64, kMaxN = 1024;
// Axis lengths (intervals) with a register-engine split: the powers of two 64..1024 and the
// 3 * 2^k / 5^2 * 2^k lengths 96, 200, 384.
constexpr bool reg_len(long long N) {
    return (N >= kMinN && N <= kMaxN && (N & (N - 1)) == 0) || N == 96 || N == 200 || N == 384;
}
// Columns per tile of the register engine (kept in sync with fft2.cuh's TileCC).  At N = 1024 a thread
// holds 32 values per FFT step and only 2 blocks fit per SM, so the tile is 4 columns wide in both
// precisions: twice the blocks of 8 columns (half the groups idle in the FFT steps, none in the loads,
// unpacking and stores), measured 25 % faster on the 1024^2 step, which has only 1024 lines per pass.
// For N = 200 (10 x 20) and 384 (16 x 24) a 16-column tile leaves 16 groups for 20 or 24 step-1 owners,
// so half the threads hold two owners; 8 columns (32 groups) give every thread at most one owner per
// step, which halves the step-1 registers (measured: a 384^2 instance's step 0.143 -> 0.086 ms, 200^2
// 0.090 -> 0.057 ms, and fewer spills in the batched kernels, whose arguments sit in shared memory).
constexpr int cc_for(bool f64, int N) { return N >= 1024 ? 4 : ((f64 || N == 200 || N == 384) ? 8 : 16); }
template <typename T, int N> cudaError_t col2_launch(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s);
template <typename T, int N> cudaError_t x2_launch(const XArgs<T>& a, int mode, dim3 grid, cudaStream_t s);
template <typename T, int N> cudaError_t prepare2();
template <typename T, int N> cudaError_t adj_col_launch(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s);
template <typename T, int N> cudaError_t adj_x_launch(const XArgs<T>& a, dim3 grid, cudaStream_t s);
template <typename T, int N> cudaError_t prepare_adj();
}  // namespace v2

// Per-launch array overrides used by the checkpointed forward recomputation.
struct StepSave {
    void* F[4];       // F(f_u), F(f_a), F(f_b), F(f_c) of the step
    void* stage[4];   // physical u, a, b, c of the step (internal layout)
};

// Adjoint workspace layout (caller-provided buffer).
struct AdjLayout {
    int64_t nsteps = 0, K = 0, nseg = 0;
    size_t off_Ub = 0, off_Cb = 0, off_Bb = 0, off_Ab = 0, off_ckpt = 0, off_seg = 0, off_grad = 0, bytes = 0;
    size_t fld = 0;   // bytes of one S-species internal array
};
AdjLayout adj_layout(const Plan& p, int64_t nsteps, int64_t K);
template <typename T> cudaError_t launch_run_checkpointed(Plan& p, void* u, double t0, int64_t nsteps, int64_t K,
                                                          char* aws, const AdjLayout& L, cudaStream_t s);
template <typename T> cudaError_t launch_adjoint(Plan& p, double t0, int64_t nsteps, int64_t K, char* aws,
                                                 const AdjLayout& L, const void* dLduT, void* dLdu0, cudaStream_t s);
cudaError_t launch_set_clock(Plan& p, double t0, cudaStream_t s, long long k0 = 0);

int kernels_per_step(const Plan& p);
// Schedule of the shared-memory engine's axes: tile width cc and the order of the radix stages
// (rule 0 as factored, 1 reversed, 2 ascending, 3 descending); rebuilds the host permutation tables
// (uploaded by the next bind).  Returns false when the rule gives the same order as an earlier rule.
bool apply_schedule(Plan* p, int cc, int rule);
bool has_generic_axis(const Plan& p);

// Plan construction and binding shared by the single-instance and batched C ABI.
int create_plan(Plan** out, const sfrd_grid* g, int bc, const double* alpha, const double* kappa, double dt,
                int dtype, const sfrd_reaction* re);
int bind_plan(Plan* p, void* ws, size_t bytes, void* stream);
int cuda_fail(cudaError_t e, const char* where);

}  // namespace sfrd
