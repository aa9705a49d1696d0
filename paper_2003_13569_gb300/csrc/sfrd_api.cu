// C ABI: plan construction (validation, FP64 tables, workspace layout), binding,
// and the load / advance / store sequencing with a captured CUDA graph per step.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <algorithm>
#include <cstdio>
#include "sfrd_internal.h"

namespace sfrd {

static thread_local std::string g_last_error;

int cuda_fail(cudaError_t e, const char* where) {
    g_last_error = std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return SFRD_ECUDA;
}

#define SFRD_CUDA(call)                                      \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
    } while (0)

__global__ void set_clock_kernel(Clock* c, double t0, long long k0) {
    c->t0 = t0;
    c->k = k0;
}

cudaError_t launch_set_clock(Plan& p, double t0, cudaStream_t s, long long k0) {
    set_clock_kernel<<<1, 1, 0, s>>>(reinterpret_cast<Clock*>(p.ws + p.off_clock), t0, k0);
    return cudaGetLastError();
}

int kernels_per_step(const Plan& p) { return p.dim == 3 ? 16 : 8; }   // 1D: x pass + combine per stage

// cos and sin of 2 pi k / M with exact octant reduction in long double.
static void cos_sin_2pi(long long k, long long M, double& c, double& s) {
    long long r = k % M;
    if (r < 0) r += M;
    const long long q = (4 * r) / M;          // quadrant
    const long long rem = 4 * r - q * M;       // angle within quadrant = (pi/2) rem / M
    long double c0, s0;
    const long double half_pi = 1.57079632679489661923132169163975144L;
    if (2 * rem <= M) {
        const long double th = half_pi * (long double)rem / (long double)M;
        c0 = cosl(th);
        s0 = sinl(th);
    } else {
        const long double th = half_pi * (long double)(M - rem) / (long double)M;
        c0 = sinl(th);
        s0 = cosl(th);
    }
    long double cc, ss;
    switch (q) {
        case 0: cc = c0; ss = s0; break;
        case 1: cc = -s0; ss = c0; break;
        case 2: cc = -c0; ss = -s0; break;
        default: cc = s0; ss = -c0; break;
    }
    c = (double)cc;
    s = (double)ss;
}

// Mixed-radix factorisation: 8s, a 4 (or 4*4 in place of 8*2), then 3s and 5s.
static bool factor(int M, std::vector<int>& r) {
    r.clear();
    int m = M, k2 = 0;
    while (m % 2 == 0) { m /= 2; ++k2; }
    int n8 = k2 / 3, rem = k2 % 3;
    if (rem == 1 && n8 > 0) { --n8; r.push_back(4); r.push_back(4); }
    for (int i = 0; i < n8; ++i) r.push_back(8);
    if (rem == 2) r.push_back(4);
    if (rem == 1 && k2 == 1) r.push_back(2);
    while (m % 3 == 0) { m /= 3; r.push_back(3); }
    while (m % 5 == 0) { m /= 5; r.push_back(5); }
    return m == 1 && (int)r.size() <= kMaxStages;  // (M <= 2048: at most 4 stages of 8 plus small factors)
}

// Slot of extension index k after the in-place DIF with radices r[0..s-1]:
// slot = sum_t d_t * M / (r_0 ... r_t), d_t the mixed-radix digits of k (least
// significant first, base r_0, r_1, ...).
static void dif_perm(int M, const std::vector<int>& r, std::vector<int>& perm) {
    perm.assign(M, 0);
    for (int k = 0; k < M; ++k) {
        int kk = k, pos = 0, w = M;
        for (int R : r) {
            const int d = kk % R;
            kk /= R;
            w /= R;
            pos += d * w;
        }
        perm[k] = pos;
    }
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static int unknowns(int bc, long long N) {
    return bc == SFRD_BC_PERIODIC ? (int)N : (bc == SFRD_BC_DIRICHLET ? (int)N - 1 : (int)N + 1);
}

// Workspace layout (byte offsets) for the plan's coefficient mode.
static void layout_workspace(Plan* p) {
    const int S = p->S;
    const size_t E = p->esize, fld = (size_t)S * p->plane * E;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t at = o; o = align_up(o + bytes, 256); return at; };
    p->off_W = take(fld);
    p->off_W2 = take(fld);
    p->off_U = take(fld);
    p->off_F1 = take(fld);
    p->off_F2 = take(fld);
    p->off_F3 = take(fld);
    if (p->coef_mode == SFRD_COEF_RATIONAL) {
        p->off_CQ = p->off_CR = 0;
        p->off_CL = take((size_t)(p->cl_shared ? 1 : S) * p->plane * E);
    } else {
        p->off_CQ = take(2 * fld);
        p->off_CR = take(4 * fld);
        p->off_CL = 0;
    }
    p->off_D = take((size_t)S * p->dense * E);
    p->off_clock = take(sizeof(Clock));
    p->off_flag = take(sizeof(int));
    for (int d = 0; d < 3; ++d) {
        p->off_tw[d] = take((size_t)p->M[d] * 2 * E);
        p->off_perm[d] = take((size_t)p->M[d] * sizeof(int));
        p->off_lam[d] = take(p->lam[d].size() * sizeof(double));
    }
    p->ws_bytes = o;
}

int create_plan(Plan** out, const sfrd_grid* g, int bc, const double* alpha, const double* kappa, double dt,
                  int dtype, const sfrd_reaction* re) {
    if (!out || !g || !alpha || !kappa || !re) return SFRD_EINVAL;
    *out = nullptr;
    if (bc < 0 || bc > 2 || (dtype != SFRD_F32 && dtype != SFRD_F64)) return SFRD_EINVAL;
    if (!(dt > 0.0) || !std::isfinite(dt)) return SFRD_EINVAL;
    if (g->dim < 1 || g->dim > 3) return SFRD_EINVAL;
    if (re->nspecies < 1 || re->nspecies > 2) return SFRD_EINVAL;
    const int S = re->nspecies;
    for (int s = 0; s < S; ++s) {
        if (!(alpha[s] > 1.0 && alpha[s] <= 2.0)) return SFRD_EINVAL;   // Eq. 1: 1 < alpha <= 2
        if (!(kappa[s] >= 0.0) || !std::isfinite(kappa[s])) return SFRD_EINVAL;
    }
    for (int d = 0; d < g->dim; ++d) {
        if (g->N[d] < 2) return SFRD_EINVAL;
        if (!(g->hi[d] > g->lo[d]) || !std::isfinite(g->hi[d] - g->lo[d])) return SFRD_EINVAL;
    }
    switch (re->kind) {
        case SFRD_REACT_NONE:
        case SFRD_REACT_LINEAR:
            break;
        case SFRD_REACT_FHN:
        case SFRD_REACT_GRAY_SCOTT:
        case SFRD_REACT_SCHNAKENBERG:
        case SFRD_REACT_GIERER_MEINHARDT:
            if (S != 2) return SFRD_EINVAL;
            break;
        case SFRD_REACT_HUXLEY_MMS:
            if (S != 1 || g->dim != 2) return SFRD_EINVAL;
            break;
        case SFRD_REACT_FISHER_MMS:
            if (S != 1 || g->dim != 1) return SFRD_EINVAL;
            break;
        default:
            return SFRD_EINVAL;
    }

    Plan* p = new (std::nothrow) Plan();
    if (!p) return SFRD_EINVAL;
    p->dim = g->dim;
    p->bc = bc;
    p->dtype = dtype;
    p->S = S;
    p->esize = dtype == SFRD_F32 ? 4 : 8;
    p->dt = dt;
    for (int s = 0; s < S; ++s) {
        p->alpha[s] = alpha[s];
        p->kappa[s] = kappa[s];
    }
    for (int d = 0; d < 3; ++d) {
        if (d < g->dim) {
            p->Nint[d] = g->N[d];
            p->lo[d] = g->lo[d];
            p->hi[d] = g->hi[d];
            p->n[d] = unknowns(bc, g->N[d]);
            const long long N = g->N[d];
            const long long M = bc == SFRD_BC_PERIODIC ? N : 2 * N;
            // the register engine's lengths (powers of two up to 1024, and 96, 200, 384) take tables of
            // length M; other lengths need a {2,3,5}-smooth M <= 1024 for the shared-memory engine
            const bool regok = v2::reg_len(N);
            if ((!regok && M > kMaxFFT) || !factor((int)M, p->radix[d])) {
                delete p;
                return SFRD_EUNSUPPORTED;
            }
            p->M[d] = (int)M;
        } else {
            p->Nint[d] = 1;
            p->n[d] = 1;
            p->M[d] = 1;
        }
    }
    // register FFT engine for power-of-two lengths (SFRD_ENGINE=generic forces the shared-memory engine)
    {
        const char* eng = std::getenv("SFRD_ENGINE");
        const bool generic = eng && std::strcmp(eng, "generic") == 0;
        for (int d = 0; d < g->dim; ++d) {
            const long long N = p->Nint[d];
            p->v2[d] = !generic && v2::reg_len(N);
        }
    }
    p->pitch = (p->n[0] + 3) / 4 * 4;
    p->plane = (long long)p->n[2] * p->n[1] * p->pitch;
    p->dense = (long long)p->n[2] * p->n[1] * p->n[0];
    // the passes index within one array (S planes) with 32-bit element offsets
    if ((unsigned long long)S * (unsigned long long)p->plane >= (1ull << 32)) {
        delete p;
        return SFRD_EUNSUPPORTED;
    }

    // reaction parameters (host-side constants of the manufactured source)
    p->re.kind = re->kind;
    p->re.S = S;
    for (int i = 0; i < 8; ++i) p->re.p[i] = re->p[i];
    p->re.off[0] = re->offset[0];
    p->re.off[1] = re->offset[1];
    p->re.c[0] = p->re.c[1] = 0.0;
    if (re->kind == SFRD_REACT_SCHNAKENBERG) {
        // the reaction at the offset: zero at the homogeneous steady state, so that the kernels add only
        // terms of the size of the perturbation (see reaction.cuh)
        const double u0 = re->offset[0], v0 = re->offset[1];
        p->re.c[0] = re->p[1] - u0 + u0 * u0 * v0;
        p->re.c[1] = re->p[2] - u0 * u0 * v0;
    }
    if (re->kind == SFRD_REACT_FISHER_MMS) {
        const double a = alpha[0], k = kappa[0];
        p->re.p[0] = k / 4.0 * 3.0 * std::pow(2.0 * M_PI, a);
        p->re.p[1] = k / 4.0 * std::pow(6.0 * M_PI, a);
    }
    if (re->kind == SFRD_REACT_HUXLEY_MMS) {
        const double a = alpha[0], k = kappa[0], pi2 = M_PI * M_PI;
        p->re.p[0] = a;
        p->re.p[1] = k / 16.0 * 9.0 * std::pow(8.0 * pi2, a / 2);
        p->re.p[2] = k / 16.0 * 3.0 * std::pow(40.0 * pi2, a / 2);
        p->re.p[3] = k / 16.0 * 3.0 * std::pow(40.0 * pi2, a / 2);
        p->re.p[4] = k / 16.0 * std::pow(72.0 * pi2, a / 2);
    }

    // FP64 tables: eigenvalues (Section 3.1), twiddles omega_M^k, DIF slot permutation
    for (int d = 0; d < 3; ++d) {
        if (d >= g->dim) {        // absent axis: one mode with eigenvalue 0, identity transform
            p->lam[d].assign(1, 0.0);
            p->tw64[d] = {1.0, 0.0};
            p->tw32[d] = {1.0f, 0.0f};
            p->perm[d].assign(1, 0);
            continue;
        }
        const long long N = p->Nint[d];
        const double h = (p->hi[d] - p->lo[d]) / (double)N;
        p->lam[d].resize(p->n[d]);
        for (int i = 0; i < p->n[d]; ++i) {
            double c, s;
            if (bc == SFRD_BC_PERIODIC) cos_sin_2pi(i, 2 * N, c, s);                    // sin(pi k / N)
            else cos_sin_2pi(i + (bc == SFRD_BC_DIRICHLET ? 1 : 0), 4 * N, c, s);      // sin(n pi / (2N))
            const double s2 = s * s;
            p->lam[d][i] = 4.0 * s2 / (h * h * (1.0 - s2 / 3.0));
        }
        const int M = p->M[d];
        p->tw64[d].resize(2 * M);
        p->tw32[d].resize(2 * M);
        for (int k = 0; k < M; ++k) {
            double c, s;
            cos_sin_2pi(k, M, c, s);
            p->tw64[d][2 * k] = c;
            p->tw64[d][2 * k + 1] = -s;
            p->tw32[d][2 * k] = (float)c;
            p->tw32[d][2 * k + 1] = (float)-s;
        }
        dif_perm(M, p->radix[d], p->perm[d]);
    }

    // tile width: the widest tile that still gives >= 2 blocks per SM on the smallest pass
    const int cands32[3] = {16, 8, 4}, cands64[3] = {8, 4, 2};
    const int* cands = dtype == SFRD_F32 ? cands32 : cands64;
    p->CC = cands[2];
    for (int i = 0; i < 3; ++i) {
        const int cc = cands[i];
        const int xw = S == 2 ? cc : 2 * cc;
        const long long rows = (long long)p->n[1] * p->n[2];
        const long long xblocks = (rows + xw - 1) / xw;
        const long long sblocks = (long long)((p->pitch + xw - 1) / xw) * (p->dim == 3 ? p->n[1] : 1);
        if (xblocks >= 304 && sblocks >= 304) {
            p->CC = cc;
            break;
        }
    }

    {
        const char* dbg = std::getenv("SFRD_DEBUG_CHECKS");
        p->debug_checks = dbg && *dbg && std::strcmp(dbg, "0") != 0;
    }
    layout_workspace(p);
    *out = p;
    return SFRD_OK;
}

// ---- schedule of the shared-memory engine and its autotuner ----------------------------

bool has_generic_axis(const Plan& p) {
    for (int d = 0; d < p.dim; ++d)
        if (!p.v2[d]) return true;
    return false;
}

bool apply_schedule(Plan* p, int cc, int rule) {
    p->CC = cc;
    bool fresh = false;
    for (int d = 0; d < p->dim; ++d) {
        if (p->v2[d]) continue;
        std::vector<int> r;
        factor(p->M[d], r);
        std::vector<int> base = r;
        if (rule == 1) std::reverse(r.begin(), r.end());
        if (rule == 2) std::stable_sort(r.begin(), r.end());
        if (rule == 3) std::stable_sort(r.begin(), r.end(), [](int x, int y) { return x > y; });
        // a rule is new for this axis unless an earlier rule (0 .. rule-1) gives the same order
        bool seen = false;
        for (int q = 0; q < rule && !seen; ++q) {
            std::vector<int> o = base;
            if (q == 1) std::reverse(o.begin(), o.end());
            if (q == 2) std::stable_sort(o.begin(), o.end());
            seen = o == r;
        }
        fresh = fresh || !seen;
        p->radix[d] = r;
        dif_perm(p->M[d], p->radix[d], p->perm[d]);
    }
    p->sched_rule = rule;
    return rule == 0 || fresh;
}

// Autotuner cache: a text file (path in SFRD_AUTOTUNE_CACHE) of lines "<key> <cc> <rule>"; the last
// line with a key wins.
static std::string schedule_key(const Plan& p) {
    int dev = 0;
    cudaDeviceProp prop{};
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) prop.name[0] = 0;
    std::string name(prop.name);
    for (char& ch : name)
        if (ch == ' ') ch = '_';
    char buf[256];
    std::snprintf(buf, sizeof(buf), "plan:d%d:N%lldx%lldx%lld:bc%d:dt%d:S%d:%s", p.dim, (long long)p.Nint[0],
                  (long long)p.Nint[1], (long long)p.Nint[2], p.bc, p.dtype, p.S, name.c_str());
    return buf;
}

static bool cache_lookup(const std::string& key, int* cc, int* rule) {
    const char* path = std::getenv("SFRD_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    std::FILE* f = std::fopen(path, "r");
    if (!f) return false;
    char k[256];
    int a = 0, b = 0;
    bool hit = false;
    while (std::fscanf(f, "%255s %d %d", k, &a, &b) == 3)
        if (key == k) {
            *cc = a;
            *rule = b;
            hit = true;
        }
    std::fclose(f);
    return hit;
}

static void cache_store(const std::string& key, int cc, int rule) {
    const char* path = std::getenv("SFRD_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    std::FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "%s %d %d\n", key.c_str(), cc, rule);
    std::fclose(f);
}

AdjLayout adj_layout(const Plan& p, int64_t nsteps, int64_t K) {
    AdjLayout L;
    L.nsteps = nsteps;
    L.K = K;
    L.nseg = (nsteps + K - 1) / K;
    L.fld = align_up((size_t)p.S * p.plane * p.esize, 256);
    size_t o = 0;
    L.off_Ub = o; o += L.fld;
    L.off_Cb = o; o += L.fld;
    L.off_Bb = o; o += L.fld;
    L.off_Ab = o; o += L.fld;
    L.off_ckpt = o; o += (size_t)L.nseg * L.fld;
    L.off_seg = o; o += (size_t)K * 9 * L.fld;
    L.off_grad = o; o += 256;
    L.bytes = o;
    return L;
}

static bool adjoint_capable(const Plan& p) {
    if (p.coef_mode == SFRD_COEF_RATIONAL) return false;   // the adjoint differentiates the stored arrays
    for (int d = 0; d < p.dim; ++d)
        if (!p.v2[d]) return false;
    return true;
}

static void drop_graph(Plan* p) {
    if (p->step_exec) cudaGraphExecDestroy(p->step_exec);
    if (p->step_graph) cudaGraphDestroy(p->step_graph);
    p->step_exec = nullptr;
    p->step_graph = nullptr;
}

int bind_plan(Plan* p, void* ws, size_t bytes, void* stream) {
    if (!ws || bytes < p->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255u)) return SFRD_ENOWS;
    drop_graph(p);
    p->ws = static_cast<char*>(ws);
    p->stream = static_cast<cudaStream_t>(stream);
    p->loaded = false;
    if (!p->cap_stream) SFRD_CUDA(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
    cudaStream_t s = p->stream;
    const size_t E = p->esize;
    for (int d = 0; d < 3; ++d) {
        const void* tw = p->dtype == SFRD_F32 ? (const void*)p->tw32[d].data() : (const void*)p->tw64[d].data();
        SFRD_CUDA(cudaMemcpyAsync(p->ws + p->off_tw[d], tw, (size_t)p->M[d] * 2 * E, cudaMemcpyHostToDevice, s));
        SFRD_CUDA(cudaMemcpyAsync(p->ws + p->off_perm[d], p->perm[d].data(), (size_t)p->M[d] * sizeof(int),
                                  cudaMemcpyHostToDevice, s));
        SFRD_CUDA(cudaMemcpyAsync(p->ws + p->off_lam[d], p->lam[d].data(), p->lam[d].size() * sizeof(double),
                                  cudaMemcpyHostToDevice, s));
    }
    const size_t fld = (size_t)p->S * p->plane * E;
    SFRD_CUDA(cudaMemsetAsync(p->ws + p->off_W, 0, 6 * fld, s));   // W, W2, U, F1, F2, F3 (padding stays 0)
    if (p->dtype == SFRD_F32) {
        SFRD_CUDA(prepare_kernels<float>(*p));
        SFRD_CUDA(launch_coef_init<float>(*p, s));
    } else {
        SFRD_CUDA(prepare_kernels<double>(*p));
        SFRD_CUDA(launch_coef_init<double>(*p, s));
    }
    SFRD_CUDA(launch_set_clock(*p, 0.0, s));
    // pageable sources: make sure the uploads are complete before the host vectors can change
    SFRD_CUDA(cudaStreamSynchronize(s));
    return SFRD_OK;
}

static cudaError_t step_direct(Plan* p, cudaStream_t s) {
    return p->dtype == SFRD_F32 ? launch_step<float>(*p, s) : launch_step<double>(*p, s);
}

static int ensure_graph(Plan* p) {
    if (p->step_exec) return SFRD_OK;
    SFRD_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = step_direct(p, p->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(p->cap_stream, &graph);
    if (e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return cuda_fail(e, "step capture");
    }
    if (e2 != cudaSuccess) return cuda_fail(e2, "cudaStreamEndCapture");
    p->step_graph = graph;
    SFRD_CUDA(cudaGraphInstantiate(&p->step_exec, graph, 0));
    return SFRD_OK;
}

static bool use_graph() {
    const char* v = std::getenv("SFRD_NO_GRAPH");
    return !(v && v[0] == '1');
}

static int load(Plan* p, const void* u0, double t0) {
    if (!p->ws) return SFRD_ENOWS;
    if (!u0) return SFRD_EINVAL;
    SFRD_CUDA(launch_set_clock(*p, t0, p->stream));
    if (p->dtype == SFRD_F32) SFRD_CUDA(launch_load<float>(*p, u0, p->stream));
    else SFRD_CUDA(launch_load<double>(*p, u0, p->stream));
    p->loaded = true;
    return SFRD_OK;
}

// SFRD_ENONFINITE when the resident state holds a NaN or an infinity (synchronises the stream).
static int check_finite(Plan* p) {
    if (!p->ws) return SFRD_ENOWS;
    if (!p->loaded) return SFRD_ESTATE;
    SFRD_CUDA(p->dtype == SFRD_F32 ? launch_finite_check<float>(*p, p->stream)
                                   : launch_finite_check<double>(*p, p->stream));
    int flag = 0;
    SFRD_CUDA(cudaMemcpyAsync(&flag, p->ws + p->off_flag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
    SFRD_CUDA(cudaStreamSynchronize(p->stream));
    return flag ? SFRD_ENONFINITE : SFRD_OK;
}

static int advance(Plan* p, int64_t nsteps) {
    if (!p->ws) return SFRD_ENOWS;
    if (!p->loaded) return SFRD_ESTATE;
    if (nsteps < 0) return SFRD_EINVAL;
    if (nsteps == 0) return SFRD_OK;
    if (use_graph()) {
        int rc = ensure_graph(p);
        if (rc != SFRD_OK) return rc;
        for (int64_t i = 0; i < nsteps; ++i) SFRD_CUDA(cudaGraphLaunch(p->step_exec, p->stream));
    } else {
        for (int64_t i = 0; i < nsteps; ++i) SFRD_CUDA(step_direct(p, p->stream));
    }
    return p->debug_checks ? check_finite(p) : SFRD_OK;
}

static int store(Plan* p, void* u) {
    if (!p->ws) return SFRD_ENOWS;
    if (!p->loaded) return SFRD_ESTATE;
    if (!u) return SFRD_EINVAL;
    if (p->dtype == SFRD_F32) SFRD_CUDA(launch_store<float>(*p, u, p->stream));
    else SFRD_CUDA(launch_store<double>(*p, u, p->stream));
    return SFRD_OK;
}

}  // namespace sfrd

using sfrd::Plan;

struct sfrd_plan_s {
    Plan p;
};

namespace sfrd {
Plan* plan_of(sfrd_plan_t h) { return &h->p; }
}  // namespace sfrd

#define SFRD_CUDA_C(call)                                           \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return sfrd::cuda_fail(e_, #call);   \
    } while (0)

extern "C" {

int sfrd_plan(sfrd_plan_t* out, const sfrd_grid* grid, int32_t bc, const double* alpha, const double* kappa,
              double dt, int32_t dtype, const sfrd_reaction* reaction) {
    if (!out) return SFRD_EINVAL;
    *out = nullptr;
    Plan* p = nullptr;
    int rc = sfrd::create_plan(&p, grid, bc, alpha, kappa, dt, dtype, reaction);
    if (rc != SFRD_OK) return rc;
    sfrd_plan_s* h = new (std::nothrow) sfrd_plan_s();
    if (!h) {
        delete p;
        return SFRD_EINVAL;
    }
    h->p = *p;
    delete p;
    *out = h;
    return SFRD_OK;
}

int sfrd_set_coefficients(sfrd_plan_t plan, int32_t mode) {
    if (!plan) return SFRD_EINVAL;
    if (mode != SFRD_COEF_STORED && mode != SFRD_COEF_RATIONAL) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (p.ws) return SFRD_ESTATE;
    if (mode == SFRD_COEF_RATIONAL) {
        if (p.dtype != SFRD_F32 || p.scheme != SFRD_SCHEME_P13) return SFRD_EUNSUPPORTED;
        for (int d = 0; d < p.dim; ++d)
            if (!p.v2[d]) return SFRD_EUNSUPPORTED;
    }
    p.coef_mode = mode;
    p.cl_shared = mode == SFRD_COEF_RATIONAL && p.S == 2 && p.alpha[0] == p.alpha[1];
    sfrd::layout_workspace(&p);
    return SFRD_OK;
}

int sfrd_set_scheme(sfrd_plan_t plan, int32_t scheme) {
    if (!plan) return SFRD_EINVAL;
    if (scheme != SFRD_SCHEME_P13 && scheme != SFRD_SCHEME_COX_MATTHEWS) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (p.ws) return SFRD_ESTATE;
    if (scheme == SFRD_SCHEME_COX_MATTHEWS && p.coef_mode != SFRD_COEF_STORED) return SFRD_EUNSUPPORTED;
    p.scheme = scheme;
    return SFRD_OK;
}

int sfrd_autotune(sfrd_plan_t plan, int32_t steps, int32_t* chosen) {
    if (!plan || steps < 1) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!p.ws) return SFRD_ENOWS;
    int best_cc = p.CC, best_rule = p.sched_rule;
    if (sfrd::has_generic_axis(p)) {
        const std::string key = sfrd::schedule_key(p);
        if (!sfrd::cache_lookup(key, &best_cc, &best_rule)) {
            const int c32[3] = {16, 8, 4}, c64[3] = {8, 4, 2};
            const int* cands = p.dtype == SFRD_F32 ? c32 : c64;
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            SFRD_CUDA_C(cudaEventCreate(&e0));
            SFRD_CUDA_C(cudaEventCreate(&e1));
            float best = -1.0f;
            int rc = SFRD_OK;
            for (int i = 0; i < 3 && rc == SFRD_OK; ++i) {
                for (int rule = 0; rule < 4 && rc == SFRD_OK; ++rule) {
                    if (!sfrd::apply_schedule(&p, cands[i], rule)) continue;
                    rc = sfrd::bind_plan(&p, p.ws, p.ws_bytes, p.stream);
                    if (rc != SFRD_OK) break;
                    cudaError_t e = sfrd::step_direct(&p, p.stream);   // warm-up
                    if (e == cudaSuccess) e = cudaEventRecord(e0, p.stream);
                    for (int k = 0; k < steps && e == cudaSuccess; ++k) e = sfrd::step_direct(&p, p.stream);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, p.stream);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float ms = 0;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                    if (e != cudaSuccess) {
                        rc = sfrd::cuda_fail(e, "sfrd_autotune");
                        break;
                    }
                    if (best < 0 || ms < best) {
                        best = ms;
                        best_cc = cands[i];
                        best_rule = rule;
                    }
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (rc != SFRD_OK) return rc;
            sfrd::cache_store(key, best_cc, best_rule);
        }
        sfrd::apply_schedule(&p, best_cc, best_rule);
        const int rc = sfrd::bind_plan(&p, p.ws, p.ws_bytes, p.stream);   // uploads the chosen tables
        if (rc != SFRD_OK) return rc;
    }
    if (chosen) {
        chosen[0] = best_cc;
        chosen[1] = best_rule;
    }
    return SFRD_OK;
}

int sfrd_workspace_bytes(sfrd_plan_t plan, size_t* bytes) {
    if (!plan || !bytes) return SFRD_EINVAL;
    *bytes = plan->p.ws_bytes;
    return SFRD_OK;
}

int sfrd_get_info(sfrd_plan_t plan, sfrd_info* info) {
    if (!plan || !info) return SFRD_EINVAL;
    const Plan& p = plan->p;
    std::memset(info, 0, sizeof(*info));
    info->dim = p.dim;
    info->bc = p.bc;
    info->dtype = p.dtype;
    info->nspecies = p.S;
    for (int d = 0; d < 3; ++d) {
        info->n[d] = d < p.dim ? p.n[d] : 1;
        info->fft_len[d] = d < p.dim ? p.M[d] : 1;
    }
    info->dof = p.dense * p.S;
    info->kernels_per_step = sfrd::kernels_per_step(p);
    info->workspace_bytes = p.ws_bytes;
    return SFRD_OK;
}

int sfrd_bind(sfrd_plan_t plan, void* workspace, size_t bytes, void* stream) {
    if (!plan) return SFRD_EINVAL;
    return sfrd::bind_plan(&plan->p, workspace, bytes, stream);
}

int sfrd_load(sfrd_plan_t plan, const void* u0, double t0) {
    if (!plan) return SFRD_EINVAL;
    return sfrd::load(&plan->p, u0, t0);
}

int sfrd_advance(sfrd_plan_t plan, int64_t nsteps) {
    if (!plan) return SFRD_EINVAL;
    return sfrd::advance(&plan->p, nsteps);
}

int sfrd_check_finite(sfrd_plan_t plan) {
    if (!plan) return SFRD_EINVAL;
    return sfrd::check_finite(&plan->p);
}

int sfrd_store(sfrd_plan_t plan, void* u) {
    if (!plan) return SFRD_EINVAL;
    return sfrd::store(&plan->p, u);
}

int sfrd_run(sfrd_plan_t plan, void* u, double t0, int64_t nsteps) {
    if (!plan) return SFRD_EINVAL;
    if (nsteps < 0) return SFRD_EINVAL;
    int rc = sfrd::load(&plan->p, u, t0);
    if (rc != SFRD_OK) return rc;
    rc = sfrd::advance(&plan->p, nsteps);
    if (rc != SFRD_OK) return rc;
    return sfrd::store(&plan->p, u);
}

int sfrd_step(sfrd_plan_t plan, void* u, double t) { return sfrd_run(plan, u, t, 1); }

int sfrd_run_host(sfrd_plan_t plan, const void* u_in, void* u_out, double t0, int64_t nsteps) {
    if (!plan || !u_in || !u_out) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!p.ws) return SFRD_ENOWS;
    const size_t bytes = (size_t)p.S * p.dense * p.esize;
    void* D = p.ws + p.off_D;
    cudaError_t e = cudaMemcpyAsync(D, u_in, bytes, cudaMemcpyHostToDevice, p.stream);
    if (e != cudaSuccess) return sfrd::cuda_fail(e, "cudaMemcpyAsync(H2D)");
    int rc = sfrd_run(plan, D, t0, nsteps);
    if (rc != SFRD_OK) return rc;
    e = cudaMemcpyAsync(u_out, D, bytes, cudaMemcpyDeviceToHost, p.stream);
    if (e != cudaSuccess) return sfrd::cuda_fail(e, "cudaMemcpyAsync(D2H)");
    e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return sfrd::cuda_fail(e, "cudaStreamSynchronize");
    return SFRD_OK;
}

int sfrd_forward(sfrd_plan_t plan, const void* u, void* uhat) {
    if (!plan || !u || !uhat) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!p.ws) return SFRD_ENOWS;
    cudaError_t e = p.dtype == SFRD_F32 ? sfrd::launch_forward<float>(p, u, uhat, p.stream)
                                        : sfrd::launch_forward<double>(p, u, uhat, p.stream);
    return e == cudaSuccess ? SFRD_OK : sfrd::cuda_fail(e, "sfrd_forward");
}

int sfrd_inverse(sfrd_plan_t plan, const void* uhat, void* u) {
    if (!plan || !u || !uhat) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!p.ws) return SFRD_ENOWS;
    cudaError_t e = p.dtype == SFRD_F32 ? sfrd::launch_inverse<float>(p, uhat, u, p.stream)
                                        : sfrd::launch_inverse<double>(p, uhat, u, p.stream);
    return e == cudaSuccess ? SFRD_OK : sfrd::cuda_fail(e, "sfrd_inverse");
}

int sfrd_coefficients(sfrd_plan_t plan, int32_t which, void* out) {
    if (!plan || !out || which < 0 || which > 5) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!p.ws) return SFRD_ENOWS;
    cudaError_t e = p.dtype == SFRD_F32 ? sfrd::launch_coef_copy<float>(p, which, out, p.stream)
                                        : sfrd::launch_coef_copy<double>(p, which, out, p.stream);
    return e == cudaSuccess ? SFRD_OK : sfrd::cuda_fail(e, "sfrd_coefficients");
}

int sfrd_profile_step(sfrd_plan_t plan, int32_t cap, float* ms, int32_t* kind) {
    if (!plan || !ms || !kind || cap < 1) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!p.ws) return SFRD_ENOWS;
    if (!p.loaded) return SFRD_ESTATE;
    const int n = sfrd::kernels_per_step(p) < cap ? sfrd::kernels_per_step(p) : cap;
    std::vector<cudaEvent_t> ev(n + 1, nullptr);
    std::vector<int> kinds(n, -1);
    for (auto& e : ev) SFRD_CUDA_C(cudaEventCreate(&e));
    cudaError_t e = p.dtype == SFRD_F32 ? sfrd::launch_step_profiled<float>(p, p.stream, ev.data(), kinds.data(), n)
                                        : sfrd::launch_step_profiled<double>(p, p.stream, ev.data(), kinds.data(), n);
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[n]);
    for (int i = 0; i < n && e == cudaSuccess; ++i) {
        e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
        kind[i] = kinds[i];
    }
    for (auto& x : ev) cudaEventDestroy(x);
    return e == cudaSuccess ? SFRD_OK : sfrd::cuda_fail(e, "sfrd_profile_step");
}

int sfrd_adjoint_workspace_bytes(sfrd_plan_t plan, int64_t nsteps, int64_t ckpt_every, size_t* bytes) {
    if (!plan || !bytes || nsteps < 1 || ckpt_every < 1) return SFRD_EINVAL;
    if (!sfrd::adjoint_capable(plan->p)) return SFRD_EUNSUPPORTED;
    *bytes = sfrd::adj_layout(plan->p, nsteps, ckpt_every).bytes;
    return SFRD_OK;
}

int sfrd_run_checkpointed(sfrd_plan_t plan, void* u, double t0, int64_t nsteps, int64_t ckpt_every, void* adj_ws,
                          size_t adj_bytes) {
    if (!plan || !u || nsteps < 1 || ckpt_every < 1) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!sfrd::adjoint_capable(p)) return SFRD_EUNSUPPORTED;
    if (!p.ws) return SFRD_ENOWS;
    const sfrd::AdjLayout L = sfrd::adj_layout(p, nsteps, ckpt_every);
    if (!adj_ws || adj_bytes < L.bytes || (reinterpret_cast<uintptr_t>(adj_ws) & 255u)) return SFRD_ENOWS;
    cudaError_t e = p.dtype == SFRD_F32
        ? sfrd::launch_run_checkpointed<float>(p, u, t0, nsteps, ckpt_every, static_cast<char*>(adj_ws), L, p.stream)
        : sfrd::launch_run_checkpointed<double>(p, u, t0, nsteps, ckpt_every, static_cast<char*>(adj_ws), L, p.stream);
    if (e != cudaSuccess) return sfrd::cuda_fail(e, "sfrd_run_checkpointed");
    p.loaded = true;
    return SFRD_OK;
}

int sfrd_adjoint(sfrd_plan_t plan, double t0, int64_t nsteps, int64_t ckpt_every, void* adj_ws, size_t adj_bytes,
                 const void* dLduT, void* dLdu0, double* dLdalpha, double* dLdkappa, double* dLdparams) {
    if (!plan || !dLduT || !dLdu0 || nsteps < 1 || ckpt_every < 1) return SFRD_EINVAL;
    Plan& p = plan->p;
    if (!sfrd::adjoint_capable(p)) return SFRD_EUNSUPPORTED;
    if (!p.ws) return SFRD_ENOWS;
    const sfrd::AdjLayout L = sfrd::adj_layout(p, nsteps, ckpt_every);
    if (!adj_ws || adj_bytes < L.bytes || (reinterpret_cast<uintptr_t>(adj_ws) & 255u)) return SFRD_ENOWS;
    char* aws = static_cast<char*>(adj_ws);
    cudaError_t e = p.dtype == SFRD_F32
        ? sfrd::launch_adjoint<float>(p, t0, nsteps, ckpt_every, aws, L, dLduT, dLdu0, p.stream)
        : sfrd::launch_adjoint<double>(p, t0, nsteps, ckpt_every, aws, L, dLduT, dLdu0, p.stream);
    if (e != cudaSuccess) return sfrd::cuda_fail(e, "sfrd_adjoint");
    double g[16];
    e = cudaMemcpyAsync(g, aws + L.off_grad, sizeof(g), cudaMemcpyDeviceToHost, p.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(p.stream);
    if (e != cudaSuccess) return sfrd::cuda_fail(e, "sfrd_adjoint (gradients)");
    for (int s = 0; s < p.S; ++s) {
        if (dLdkappa) dLdkappa[s] = g[s];
        if (dLdalpha) dLdalpha[s] = g[2 + s];
    }
    if (dLdparams)
        for (int q = 0; q < 8; ++q) dLdparams[q] = q < 5 ? g[4 + q] : 0.0;
    p.loaded = false;   // the work arrays were reused
    return SFRD_OK;
}

void sfrd_destroy(sfrd_plan_t plan) {
    if (!plan) return;
    sfrd::drop_graph(&plan->p);
    if (plan->p.cap_stream) cudaStreamDestroy(plan->p.cap_stream);
    delete plan;
}

const char* sfrd_strerror(int code) {
    switch (code) {
        case SFRD_OK: return "ok";
        case SFRD_EINVAL: return "invalid argument";
        case SFRD_EUNSUPPORTED: return "unsupported problem size or dimension";
        case SFRD_ENOWS: return "workspace missing, too small or misaligned";
        case SFRD_ECUDA: return "CUDA runtime error";
        case SFRD_ENONFINITE: return "non-finite value in the state";
        case SFRD_ESTATE: return "call out of order (no state loaded)";
        default: return "unknown error";
    }
}

const char* sfrd_last_error(void) { return sfrd::g_last_error.c_str(); }

}  // extern "C"
