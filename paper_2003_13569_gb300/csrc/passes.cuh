// Transform passes of one ETDRK4-P13 step and their launchers.
//
// Internal field layout (device workspace): species-major [S][n_z][n_y][pitch],
// x contiguous, pitch = n_x rounded up to a multiple of 4 (padding held at 0).
// Spectral arrays use the same layout with mode indices in eigenvalue order.
//
// One step (Algorithm 1, restructured by linearity so that each stage needs
// one forward and one inverse separable transform per species) is four chains;
// the slow axis is z in 3D and y in 2D:
//   3D:  [middle y]  ->  [x: T_x, f, T_x]  ->  [middle y]  ->  [slow z: T_z, combine, T_z]
//   2D:                  [x: T_x, f, T_x]  ->                  [slow y: T_y, combine, T_y]
// The x pass carries the reaction (f at the stage time), the slow-axis pass
// carries the Pade-(1,3) combination of Eq. ETDRK4P13:
//   stage a:  a^ = Q13 u^ + phi F(f_u)
//   stage b:  b^ = Q13 u^ + phi F(f_a)
//   stage c:  c^ = Q13 (Q13 u^ + phi F(f_u)) + phi (2 F(f_b) - F(f_u))   [F(a) by linearity]
//   update :  u^' = R13 u^ + phi1 F(f_u) + phi2 (F(f_a) + F(f_b)) + phi3 F(f_c)
// where F = T_z T_y T_x is the unnormalised real transform of each axis and
// the inverse is F / C.  All passes run in place on the work array.
#pragma once

#include "adjgrad.cuh"
#include "coef.cuh"
#include "engine.cuh"
#include "reaction.cuh"

namespace sfrd {

// Value of the transform at unknown k from a DFT output held in slot order.
template <typename C, bool PERM>
__device__ __forceinline__ C get_one(const C* buf, int ldb, const AxisDev& ax, int k, int c) {
    using T = decltype(buf[0].x);
    C v;
    if (ax.bc == SFRD_BC_PERIODIC) {
        const int k1 = (ax.N - k) % ax.N;
        const int r0 = PERM ? __ldg(ax.perm + k) : k;
        const int r1 = PERM ? __ldg(ax.perm + k1) : k1;
        const C z0 = buf[r0 * ldb + c], z1 = buf[r1 * ldb + c];
        v.x = (T)0.5 * (z0.x + z1.x + z1.y - z0.y);
        v.y = (T)0.5 * (z0.y + z1.y + z0.x - z1.x);
        return v;
    }
    const int e = ext_index(ax.bc, k);
    const int r0 = PERM ? __ldg(ax.perm + e) : e;
    const C z = buf[r0 * ldb + c];
    if (ax.bc == SFRD_BC_DIRICHLET) {
        v.x = (T)-0.5 * z.y;
        v.y = (T)0.5 * z.x;
    } else {
        v.x = (T)0.5 * z.x;
        v.y = (T)0.5 * z.y;
    }
    return v;
}

// ---- strided-axis pass (y or z): tile = all unknowns along the axis x CC columns ----

// Body of the strided pass for tile (bx, by); smem = dynamic shared memory of the block.
template <typename T, int CC, int MODE>
__device__ __forceinline__ void col_body(const ColArgs<T>& a, int bx, int by, unsigned char* smem_raw) {
    using C = typename Cx<T>::type;
    C* buf = reinterpret_cast<C*>(smem_raw);
    constexpr int ldb = CC + 1;
    constexpr int G = kThreads / CC;
    const int tid = threadIdx.x, c = tid % CC, grp = tid / CC;
    const AxisDev& ax = a.ax;
    const int xA = bx * a.xw + c * a.cstride;
    const int xB = xA + a.bshift;
    const long long other = by;

    // load along the axis, natural order, with the odd/even extension
    {
        const bool okA = xA < a.in_xlim, okB = xB < a.in_xlim;
        const T* pA = a.in + other * a.in_sOther + xA;
        for (int i = grp; i < ax.n; i += G) {
            C z;
            z.x = okA ? pA[i * a.in_sAxis] : (T)0;
            z.y = okB ? pA[i * a.in_sAxis + a.in_offB] : (T)0;
            put_extended<C, false>(buf, ldb, ax, i, c, z);
        }
        put_extension_zeros<C, false>(buf, ldb, ax, c, grp);
    }
    __syncthreads();
    fft_dif(buf, ldb, ax, c, grp, G);

    const int items = unpack_items(ax);
    if (MODE == MODE_PLAIN) {
        const bool okA = xA < a.out_xlim, okB = xB < a.out_xlim;
        T* qA = a.out + other * a.out_sOther + xA;
        const T sc = (T)a.scale;
        for (int it = grp; it < items; it += G) {
            int k0, k1;
            C v0, v1;
            const int cnt = get_transform<C, true>(buf, ldb, ax, it, c, k0, v0, k1, v1);
            if (okA) qA[k0 * a.out_sAxis] = v0.x * sc;
            if (okB) qA[k0 * a.out_sAxis + a.out_offB] = v0.y * sc;
            if (cnt == 2) {
                if (okA) qA[k1 * a.out_sAxis] = v1.x * sc;
                if (okB) qA[k1 * a.out_sAxis + a.out_offB] = v1.y * sc;
            }
        }
        return;
    }

    // slow-axis modes: spectral combination, then the inverse along the axis
    {
        const bool okA = xA < a.in_xlim, okB = xB < a.in_xlim;
        const long long base = other * a.in_sOther + xA;
        const long long oB = a.in_offB;
        const T invC = (T)a.invC;
        for (int it = grp; it < items; it += G) {
            int ks[2];
            C vs[2];
            const int cnt = get_transform<C, true>(buf, ldb, ax, it, c, ks[0], vs[0], ks[1], vs[1]);
            for (int q = 0; q < cnt; ++q) {
                const int k = ks[q];
                const long long iA = base + k * a.in_sAxis, iB = iA + oB;
                T F[2] = {vs[q].x, vs[q].y};
                T s[2] = {0, 0};
                const bool ok[2] = {okA, okB};
                const long long ix[2] = {iA, iB};
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    if (!ok[h]) continue;
                    const long long i = ix[h];
                    if (MODE == MODE_T0) {
                        a.U[i] = F[h];
                        s[h] = F[h];
                    } else if (MODE == MODE_TA || MODE == MODE_TB) {
                        if (MODE == MODE_TA) a.F1[i] = F[h]; else a.F2[i] = F[h];
                        const T Q = a.CQ[2 * i], ph = a.CQ[2 * i + 1];
                        s[h] = Q * a.U[i] + ph * F[h];
                    } else if (MODE == MODE_TC) {
                        a.F3[i] = F[h];
                        const T Q = a.CQ[2 * i], ph = a.CQ[2 * i + 1];
                        const T f1 = a.F1[i];
                        const T ah = Q * a.U[i] + ph * f1;
                        s[h] = Q * ah + ph * ((T)2 * F[h] - f1);
                    } else {  // MODE_TD
                        const T R = a.CR[4 * i], p1 = a.CR[4 * i + 1], p2 = a.CR[4 * i + 2], p3 = a.CR[4 * i + 3];
                        const T un = R * a.U[i] + p1 * a.F1[i] + p2 * (a.F2[i] + a.F3[i]) + p3 * F[h];
                        a.U[i] = un;
                        s[h] = un;
                    }
                }
                C z;
                z.x = s[0] * invC;
                z.y = s[1] * invC;
                put_value<C, true>(buf, ldb, ax, k, c, z);
            }
        }
        put_extension_zeros<C, true>(buf, ldb, ax, c, grp);
    }
    __syncthreads();
    fft_dit(buf, ldb, ax, c, grp, G);
    {
        const bool okA = xA < a.out_xlim, okB = xB < a.out_xlim;
        T* qA = a.out + other * a.out_sOther + xA;
        for (int i = grp; i < ax.n; i += G) {
            const C v = get_one<C, false>(buf, ldb, ax, i, c);
            if (okA) qA[i * a.out_sAxis] = v.x;
            if (okB) qA[i * a.out_sAxis + a.out_offB] = v.y;
        }
    }
    if (MODE == MODE_TD && bx == 0 && by == 0 && threadIdx.x == 0) a.clock->k += 1;
}

template <typename T, int CC, int MODE>
__global__ void __launch_bounds__(kThreads) col_kernel(const ColArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    col_body<T, CC, MODE>(a, blockIdx.x, blockIdx.y, smem_raw);
}

// ---- contiguous-axis pass: tile = CC row pairs (species 0 / species 1, or two rows) ----

template <typename T, int CC, int MODE>
__device__ __forceinline__ void x_body(const XArgs<T>& a, int bx, unsigned char* smem_raw) {
    using C = typename Cx<T>::type;
    C* buf = reinterpret_cast<C*>(smem_raw);
    constexpr int ldb = CC + 1;
    constexpr int G = kThreads / CC;
    const int tid = threadIdx.x, c = tid % CC, grp = tid / CC;
    const AxisDev& ax = a.ax;
    const int n = ax.n;
    const int shiftB = (a.S == 2) ? 0 : CC;
    const int r0 = bx * (a.S == 2 ? CC : 2 * CC);

    // transposed load: consecutive threads read consecutive x of one row
    for (int q = tid; q < CC * n; q += kThreads) {
        const int cc = q / n, i = q - cc * n;
        const int rA = r0 + cc, rB = rA + shiftB;
        C z;
        z.x = rA < a.rows ? a.in[(long long)rA * a.in_pitch + i] : (T)0;
        z.y = rB < a.rows ? a.in[(long long)rA * a.in_pitch + a.in_offB + i] : (T)0;
        put_extended<C, false>(buf, ldb, ax, i, cc, z);
    }
    if (tid < CC) put_extension_zeros<C, false>(buf, ldb, ax, tid, 0);
    __syncthreads();
    fft_dif(buf, ldb, ax, c, grp, G);

    if (MODE == MODE_REACT) {
        const double t = a.clock->t0 + ((double)a.clock->k + a.stage_frac) * a.tau;
        const int items = unpack_items(ax);
        const int rA = r0 + c, rB = rA + shiftB;
        for (int it = grp; it < items; it += G) {
            int ks[2];
            C vs[2];
            const int cnt = get_transform<C, true>(buf, ldb, ax, it, c, ks[0], vs[0], ks[1], vs[1]);
            for (int q = 0; q < cnt; ++q) {
                const int k = ks[q];
                C f;
                if (a.S == 2) {
                    react2<T>(a.re, vs[q].x, vs[q].y, f.x, f.y);
                } else {
                    const double x = ax.lo + (ax.node0 + k) * ax.h;
                    const int yA = rA % a.ny, yB = rB % a.ny;
                    const double ya = a.ay.lo + (a.ay.node0 + yA) * a.ay.h;
                    const double yb = a.ay.lo + (a.ay.node0 + yB) * a.ay.h;
                    f.x = react1<T>(a.re, vs[q].x, x, ya, t);
                    f.y = react1<T>(a.re, vs[q].y, x, yb, t);
                }
                put_value<C, true>(buf, ldb, ax, k, c, f);
            }
        }
        put_extension_zeros<C, true>(buf, ldb, ax, c, grp);
        __syncthreads();
        fft_dit(buf, ldb, ax, c, grp, G);
        for (int q = tid; q < CC * n; q += kThreads) {
            const int cc = q / n, i = q - cc * n;
            const int rA2 = r0 + cc, rB2 = rA2 + shiftB;
            const C v = get_one<C, false>(buf, ldb, ax, i, cc);
            if (rA2 < a.rows) a.out[(long long)rA2 * a.out_pitch + i] = v.x;
            if (rB2 < a.rows) a.out[(long long)rA2 * a.out_pitch + a.out_offB + i] = v.y;
        }
    } else {
        for (int q = tid; q < CC * n; q += kThreads) {
            const int cc = q / n, i = q - cc * n;
            const int rA2 = r0 + cc, rB2 = rA2 + shiftB;
            const C v = get_one<C, true>(buf, ldb, ax, i, cc);
            if (rA2 < a.rows) a.out[(long long)rA2 * a.out_pitch + i] = v.x;
            if (rB2 < a.rows) a.out[(long long)rA2 * a.out_pitch + a.out_offB + i] = v.y;
        }
    }
    // keep the padding columns of internal rows at zero
    const int pad = a.out_fill - n;
    if (pad > 0) {
        for (int q = tid; q < CC * pad; q += kThreads) {
            const int cc = q / pad, i = n + (q - cc * pad);
            const int rA2 = r0 + cc, rB2 = rA2 + shiftB;
            if (rA2 < a.rows) a.out[(long long)rA2 * a.out_pitch + i] = (T)0;
            if (rB2 < a.rows) a.out[(long long)rA2 * a.out_pitch + a.out_offB + i] = (T)0;
        }
    }
}

template <typename T, int CC, int MODE>
__global__ void __launch_bounds__(kThreads) x_kernel(const XArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    x_body<T, CC, MODE>(a, blockIdx.x, smem_raw);
}

// ---- plan-time FP64 coefficient kernel (Algorithm 1, precompute lines) ----------

template <typename T>
__global__ void coef_init_kernel(const double* __restrict__ lx, const double* __restrict__ ly,
                                 const double* __restrict__ lz, int nx, int ny, int nz, int pitch,
                                 int S, double a0, double a1, double k0, double k1, double tau, int scheme,
                                 T* __restrict__ CQ, T* __restrict__ CR) {
    const long long total = (long long)S * nz * ny * pitch;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % pitch);
        long long r = idx / pitch;
        const int y = (int)(r % ny);
        r /= ny;
        const int z = (int)(r % nz);
        const int s = (int)(r / nz);
        double Q = 0, ph = 0, R = 0, p1 = 0, p2 = 0, p3 = 0;
        if (x < nx) {
            const double Lam = lx[x] + ly[y] + lz[z];           // summed eigenvalue (Eqs. E16-E22)
            const double alpha = s == 0 ? a0 : a1, kappa = s == 0 ? k0 : k1;
            const double Lf = Lam > 0.0 ? pow(Lam, 0.5 * alpha) : 0.0;   // Lambda^{alpha/2}
            const double L = kappa * tau * Lf;                  // L = kappa tau Lambda^{alpha/2}
            if (scheme == SFRD_SCHEME_COX_MATTHEWS) {
                cm_coefficients(L, tau, R, Q, ph, p1, p2, p3);
            } else {
                const double D1 = 24.0 + L * (18.0 + L * (6.0 + L));
                const double D2 = 192.0 + L * (72.0 + L * (12.0 + L));
                R = (24.0 - 6.0 * L) / D1;
                Q = 24.0 * (8.0 - L) / D2;
                ph = tau * (96.0 + L * (12.0 + L)) / D2;
                p1 = tau * (4.0 - L) / D1;
                p2 = 2.0 * tau * (4.0 + L) / D1;
                p3 = tau * (4.0 + L * (3.0 + L)) / D1;
            }
        }
        CQ[2 * idx] = (T)Q;
        CQ[2 * idx + 1] = (T)ph;
        CR[4 * idx] = (T)R;
        CR[4 * idx + 1] = (T)p1;
        CR[4 * idx + 2] = (T)p2;
        CR[4 * idx + 3] = (T)p3;
    }
}

// Rational-coefficient mode: L (or tau Lambda^{alpha/2} shared by the species) in FP64, stored in T.
template <typename T>
__global__ void coef_l_kernel(const double* __restrict__ lx, const double* __restrict__ ly,
                              const double* __restrict__ lz, int nx, int ny, int nz, int pitch, int planes,
                              bool shared, double a0, double a1, double k0, double k1, double tau,
                              T* __restrict__ CL) {
    const long long total = (long long)planes * nz * ny * pitch;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % pitch);
        long long r = idx / pitch;
        const int y = (int)(r % ny);
        r /= ny;
        const int z = (int)(r % nz);
        const int s = (int)(r / nz);
        double v = 0;
        if (x < nx) {
            const double Lam = lx[x] + ly[y] + lz[z];
            const double alpha = s == 0 ? a0 : a1, kappa = shared ? 1.0 : (s == 0 ? k0 : k1);
            v = kappa * tau * (Lam > 0.0 ? pow(Lam, 0.5 * alpha) : 0.0);
        }
        CL[idx] = (T)v;
    }
}

// Coefficient `which` evaluated from the stored L (rational mode), in T, to dense [S][nz][ny][nx].
template <typename T>
__global__ void coef_eval_kernel(const T* __restrict__ CL, bool shared, double k0, double k1, double tau, int which,
                                 int nx, int ny, int nz, int pitch, int S, T* __restrict__ out) {
    const long long total = (long long)S * nz * ny * nx;
    const long long plane = (long long)nz * ny * pitch;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % nx);
        const long long row = idx / nx;                 // s * nz * ny + (z * ny + y)
        const int s = (int)(row / ((long long)nz * ny));
        const long long j = (row - (long long)s * nz * ny) * pitch + x;
        const T L = shared ? (T)(s == 0 ? k0 : k1) * CL[j] : CL[s * plane + j];
        T Q, ph, R, p1, p2, p3;
        p13_qphi<T>(L, (T)tau, Q, ph);
        p13_rphi<T>(L, (T)tau, R, p1, p2, p3);
        const T v[6] = {R, Q, ph, p1, p2, p3};
        out[idx] = v[which];
    }
}

// which: 0 R13, 1 Q13, 2 phi, 3 phi1, 4 phi2, 5 phi3 -> dense [S][nz][ny][nx]
template <typename T>
__global__ void coef_copy_kernel(const T* __restrict__ CQ, const T* __restrict__ CR, int which, int nx,
                                 int ny, int nz, int pitch, int S, T* __restrict__ out) {
    const long long total = (long long)S * nz * ny * nx;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % nx);
        const long long row = idx / nx;
        const long long j = row * pitch + x;
        T v;
        switch (which) {
            case 0: v = CR[4 * j]; break;
            case 1: v = CQ[2 * j]; break;
            case 2: v = CQ[2 * j + 1]; break;
            case 3: v = CR[4 * j + 1]; break;
            case 4: v = CR[4 * j + 2]; break;
            default: v = CR[4 * j + 3]; break;
        }
        out[idx] = v;
    }
}

// ---- launchers -------------------------------------------------------------------

#define SFRD_TRY(x)                          \
    do {                                     \
        cudaError_t e_ = (x);                \
        if (e_ != cudaSuccess) return e_;    \
    } while (0)

template <typename T, int CC>
static cudaError_t col_launch(const ColArgs<T>& a, int mode, dim3 grid, size_t smem, cudaStream_t s) {
    void (*k)(const ColArgs<T>) = nullptr;
    switch (mode) {
        case MODE_PLAIN: k = col_kernel<T, CC, MODE_PLAIN>; break;
        case MODE_T0: k = col_kernel<T, CC, MODE_T0>; break;
        case MODE_TA: k = col_kernel<T, CC, MODE_TA>; break;
        case MODE_TB: k = col_kernel<T, CC, MODE_TB>; break;
        case MODE_TC: k = col_kernel<T, CC, MODE_TC>; break;
        default: k = col_kernel<T, CC, MODE_TD>; break;
    }
    k<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int CC>
static cudaError_t x_launch(const XArgs<T>& a, int mode, dim3 grid, size_t smem, cudaStream_t s) {
    void (*k)(const XArgs<T>) = (mode == MODE_REACT) ? x_kernel<T, CC, MODE_REACT> : x_kernel<T, CC, MODE_PLAIN>;
    k<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

// Raise the dynamic shared-memory limit of every pass kernel of one tile width
// (done once at bind time, outside any stream capture).
constexpr int kMaxDynSmem = 227 * 1024;

template <typename T, int CC>
static cudaError_t prepare_cc() {
    void (*ks[])(const ColArgs<T>) = {col_kernel<T, CC, MODE_PLAIN>, col_kernel<T, CC, MODE_T0>,
                                      col_kernel<T, CC, MODE_TA>,    col_kernel<T, CC, MODE_TB>,
                                      col_kernel<T, CC, MODE_TC>,    col_kernel<T, CC, MODE_TD>};
    for (auto k : ks) SFRD_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
    void (*xs[])(const XArgs<T>) = {x_kernel<T, CC, MODE_PLAIN>, x_kernel<T, CC, MODE_REACT>};
    for (auto k : xs) SFRD_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxDynSmem));
    return cudaSuccess;
}

template <typename T> struct CCs;
template <> struct CCs<float> { static constexpr int a = 16, b = 8, c = 4; };
template <> struct CCs<double> { static constexpr int a = 8, b = 4, c = 2; };

template <typename T>
static AxisDev axis_dev(const Plan& p, int d) {
    AxisDev ax{};
    ax.n = p.n[d];
    ax.N = (int)p.Nint[d];
    ax.M = p.M[d];
    ax.bc = p.bc;
    ax.nst = (int)p.radix[d].size();
    for (int i = 0; i < ax.nst; ++i) ax.radix[i] = p.radix[d][i];
    ax.tw = p.ws + p.off_tw[d];
    ax.perm = reinterpret_cast<const int*>(p.ws + p.off_perm[d]);
    ax.node0 = p.bc == SFRD_BC_DIRICHLET ? 1 : 0;
    ax.h = (p.hi[d] - p.lo[d]) / (double)p.Nint[d];
    ax.lo = p.lo[d];
    return ax;
}

template <typename T>
static size_t tile_smem(const Plan& p, int d) {
    return (size_t)p.M[d] * (size_t)(p.CC + 1) * 2 * sizeof(T);
}

template <typename T>
static cudaError_t dispatch_col(const Plan& p, const ColArgs<T>& a, int mode, dim3 grid, size_t smem, cudaStream_t s) {
    if (p.CC == CCs<T>::a) return col_launch<T, CCs<T>::a>(a, mode, grid, smem, s);
    if (p.CC == CCs<T>::b) return col_launch<T, CCs<T>::b>(a, mode, grid, smem, s);
    return col_launch<T, CCs<T>::c>(a, mode, grid, smem, s);
}

template <typename T>
static cudaError_t dispatch_x(const Plan& p, const XArgs<T>& a, int mode, dim3 grid, size_t smem, cudaStream_t s) {
    if (p.CC == CCs<T>::a) return x_launch<T, CCs<T>::a>(a, mode, grid, smem, s);
    if (p.CC == CCs<T>::b) return x_launch<T, CCs<T>::b>(a, mode, grid, smem, s);
    return x_launch<T, CCs<T>::c>(a, mode, grid, smem, s);
}

template <typename T>
cudaError_t prepare_kernels(const Plan& p) {
    for (int d = 0; d < p.dim; ++d) {
        if (!p.v2[d]) continue;
        switch (p.Nint[d]) {
            case 64: SFRD_TRY((v2::prepare2<T, 64>())); SFRD_TRY((v2::prepare_adj<T, 64>())); break;
            case 128: SFRD_TRY((v2::prepare2<T, 128>())); SFRD_TRY((v2::prepare_adj<T, 128>())); break;
            case 256: SFRD_TRY((v2::prepare2<T, 256>())); SFRD_TRY((v2::prepare_adj<T, 256>())); break;
            case 512: SFRD_TRY((v2::prepare2<T, 512>())); SFRD_TRY((v2::prepare_adj<T, 512>())); break;
            case 96: SFRD_TRY((v2::prepare2<T, 96>())); SFRD_TRY((v2::prepare_adj<T, 96>())); break;
            case 200: SFRD_TRY((v2::prepare2<T, 200>())); SFRD_TRY((v2::prepare_adj<T, 200>())); break;
            case 384: SFRD_TRY((v2::prepare2<T, 384>())); SFRD_TRY((v2::prepare_adj<T, 384>())); break;
            default: SFRD_TRY((v2::prepare2<T, 1024>())); SFRD_TRY((v2::prepare_adj<T, 1024>())); break;
        }
    }
    SFRD_TRY((prepare_cc<T, CCs<T>::a>()));
    SFRD_TRY((prepare_cc<T, CCs<T>::b>()));
    return prepare_cc<T, CCs<T>::c>();
}

template <typename T> static T* wsT(const Plan& p, size_t off) { return reinterpret_cast<T*>(p.ws + off); }

// Array description: base pointer, row pitch, species plane stride.
template <typename T>
struct Arr {
    const T* ptr;
    long long pitch;
    long long plane;
    int xlim;
};

template <typename T>
static Arr<T> internal_arr(const Plan& p, size_t off) {
    return Arr<T>{wsT<T>(p, off), p.pitch, p.plane, p.pitch};
}

template <typename T>
static Arr<T> dense_arr(const Plan& p, const void* ptr) {
    return Arr<T>{static_cast<const T*>(ptr), p.n[0], p.dense, p.n[0]};
}

// pair_grid: for a slow-axis pass of an FP32 two-species plan on the register engine with internal
// arrays, the lines A and B are the adjacent columns x, x + 1 of one species and the species is
// blockIdx.z (the slow-axis kernels then read and write element pairs).
template <typename T>
static bool use_pair_grid(const Plan& p, int d, const Arr<T>& in, const Arr<T>& out) {
    return sizeof(T) == 4 && p.S == 2 && p.v2[d] && d == (p.dim == 3 ? 2 : 1) &&
           in.pitch % 4 == 0 && out.pitch % 4 == 0 && in.xlim == in.pitch && out.xlim == out.pitch;
}

// Strided pass along axis d (1 = y, 2 = z) from array `in` to `out`.
template <typename T>
static ColArgs<T> col_args(const Plan& p, int d, const Arr<T>& in, const Arr<T>& out, double scale, dim3& grid,
                           bool pair_grid = false) {
    ColArgs<T> a{};
    const int ny = p.n[1];
    a.in = in.ptr;
    a.out = const_cast<T*>(out.ptr);
    const bool use2 = p.v2[d];
    const int cc = use2 ? v2::cc_for(sizeof(T) == 8, (int)p.Nint[d]) : p.CC;
    // The two real lines of a tile column: the two species at one x, or (one species, and the
    // middle axis of a 3D grid whose species planes follow one another along blockIdx.y) the
    // columns x and x + cc, so that a tile row is 2 cc consecutive values of one array row.
    const bool species_rows = p.S == 2 && d == 1 && p.dim == 3 &&
                              in.plane == (long long)p.n[2] * ny * in.pitch &&
                              out.plane == (long long)p.n[2] * ny * out.pitch;
    const bool two = p.S == 2 && !species_rows;
    a.bshift = two ? 0 : cc;
    a.xw = two ? cc : 2 * cc;
    a.in_offB = two ? in.plane : cc;
    a.out_offB = two ? out.plane : cc;
    a.cstride = 1;
    a.in_sp = a.out_sp = 0;
    const bool pairs = pair_grid && use_pair_grid<T>(p, d, in, out);
    if (species_rows || pairs) {   // lines A and B of a lane: the adjacent columns x, x + 1 (one 2-element access)
        a.bshift = 1;
        a.xw = 2 * cc;
        a.in_offB = a.out_offB = 1;
        a.cstride = 2;
    }
    if (pairs) {
        a.in_sp = in.plane;
        a.out_sp = out.plane;
    }
    int gy = 1;
    if (d == 2) {          // z in 3D: blockIdx.y = y
        a.in_sAxis = (long long)ny * in.pitch;
        a.in_sOther = in.pitch;
        a.out_sAxis = (long long)ny * out.pitch;
        a.out_sOther = out.pitch;
        gy = ny;
    } else if (p.dim == 3) {   // y in 3D: blockIdx.y = z (+ n_z * species)
        a.in_sAxis = in.pitch;
        a.in_sOther = (long long)ny * in.pitch;
        a.out_sAxis = out.pitch;
        a.out_sOther = (long long)ny * out.pitch;
        gy = p.n[2] * (species_rows ? p.S : 1);
    } else {               // y in 2D
        a.in_sAxis = in.pitch;
        a.in_sOther = 0;
        a.out_sAxis = out.pitch;
        a.out_sOther = 0;
        gy = 1;
    }
    a.in_xlim = in.xlim;
    a.out_xlim = out.xlim;
    a.scale = scale;
    double C = 1.0;
    for (int k = 0; k < p.dim; ++k) C *= (p.bc == SFRD_BC_PERIODIC) ? (double)p.Nint[k] : 0.5 * (double)p.Nint[k];
    a.invC = 1.0 / C;
    a.U = wsT<T>(p, p.off_U);
    a.F1 = wsT<T>(p, p.off_F1);
    a.F2 = wsT<T>(p, p.off_F2);
    a.F3 = wsT<T>(p, p.off_F3);
    a.CQ = wsT<T>(p, p.off_CQ);
    a.CR = wsT<T>(p, p.off_CR);
    a.CL = nullptr;
    if (p.coef_mode == SFRD_COEF_RATIONAL) {
        a.CQ = a.CR = nullptr;
        a.CL = wsT<T>(p, p.off_CL);
        for (int h = 0; h < 2; ++h) a.cl_mult[h] = p.cl_shared ? p.kappa[h] : 1.0;
        a.clB = p.cl_shared ? 0 : a.in_offB;
        a.cl_sp = p.cl_shared ? 0 : p.plane;
    }
    a.clock = reinterpret_cast<Clock*>(p.ws + p.off_clock);
    a.ax = axis_dev<T>(p, d);
    a.dim = p.dim;
    a.S = p.S;
    for (int k = 0; k < 3; ++k) {
        a.lam[k] = reinterpret_cast<const double*>(p.ws + p.off_lam[k]);
        a.nk[k] = p.n[k];
    }
    for (int k = 0; k < 2; ++k) {
        a.alpha[k] = p.alpha[p.S == 2 ? k : 0];
        a.kappa[k] = p.kappa[p.S == 2 ? k : 0];
    }
    a.tau = p.dt;
    a.scheme = p.scheme;
    const int xlim = in.xlim > out.xlim ? in.xlim : out.xlim;
    grid = dim3((xlim + a.xw - 1) / a.xw, gy, pairs ? p.S : 1);
    return a;
}

template <typename T>
static cudaError_t launch_col(const Plan& p, int d, int mode, const ColArgs<T>& a, dim3 grid, cudaStream_t s) {
    if (p.v2[d]) {
        const bool adj = mode >= MODE_ADJ_ENTRY;
        switch (p.Nint[d]) {
            case 64: return adj ? v2::adj_col_launch<T, 64>(a, mode, grid, s) : v2::col2_launch<T, 64>(a, mode, grid, s);
            case 128: return adj ? v2::adj_col_launch<T, 128>(a, mode, grid, s) : v2::col2_launch<T, 128>(a, mode, grid, s);
            case 256: return adj ? v2::adj_col_launch<T, 256>(a, mode, grid, s) : v2::col2_launch<T, 256>(a, mode, grid, s);
            case 512: return adj ? v2::adj_col_launch<T, 512>(a, mode, grid, s) : v2::col2_launch<T, 512>(a, mode, grid, s);
            case 96: return adj ? v2::adj_col_launch<T, 96>(a, mode, grid, s) : v2::col2_launch<T, 96>(a, mode, grid, s);
            case 200: return adj ? v2::adj_col_launch<T, 200>(a, mode, grid, s) : v2::col2_launch<T, 200>(a, mode, grid, s);
            case 384: return adj ? v2::adj_col_launch<T, 384>(a, mode, grid, s) : v2::col2_launch<T, 384>(a, mode, grid, s);
            default: return adj ? v2::adj_col_launch<T, 1024>(a, mode, grid, s) : v2::col2_launch<T, 1024>(a, mode, grid, s);
        }
    }
    if (mode >= MODE_ADJ_ENTRY) return cudaErrorNotSupported;
    return dispatch_col<T>(p, a, mode, grid, tile_smem<T>(p, d), s);
}

// Strided pass along axis d (1 = y, 2 = z) from array `in` to `out`.
template <typename T>
static cudaError_t run_col(const Plan& p, int d, int mode, const Arr<T>& in, const Arr<T>& out, double scale,
                           cudaStream_t s) {
    dim3 grid;
    const ColArgs<T> a = col_args<T>(p, d, in, out, scale, grid);
    return launch_col<T>(p, d, mode, a, grid, s);
}

template <typename T>
static XArgs<T> x_args(const Plan& p, const Arr<T>& in, const Arr<T>& out, int out_fill, double stage_frac,
                       dim3& grid) {
    XArgs<T> a{};
    a.in = in.ptr;
    a.out = const_cast<T*>(out.ptr);
    const bool two = p.S == 2;
    const bool use2 = p.v2[0];
    const int cc = use2 ? v2::cc_for(sizeof(T) == 8, (int)p.Nint[0]) : p.CC;
    a.S = p.S;
    a.in_pitch = in.pitch;
    a.out_pitch = out.pitch;
    a.in_offB = two ? in.plane : (long long)cc * in.pitch;
    a.out_offB = two ? out.plane : (long long)cc * out.pitch;
    a.rows = p.n[1] * p.n[2];
    a.out_fill = out_fill;
    a.ny = p.n[1];
    a.nz = p.n[2];
    a.tau = p.dt;
    a.stage_frac = stage_frac;
    a.clock = reinterpret_cast<const Clock*>(p.ws + p.off_clock);
    a.ax = axis_dev<T>(p, 0);
    a.ay = axis_dev<T>(p, 1);
    if (p.dim == 3) a.az = axis_dev<T>(p, 2);
    a.re = p.re;
    const int per = two ? cc : 2 * cc;
    grid = dim3((a.rows + per - 1) / per, 1, 1);
    return a;
}

template <typename T>
static cudaError_t launch_x(const Plan& p, int mode, const XArgs<T>& a, dim3 grid, cudaStream_t s) {
    if (p.v2[0]) {
        const bool adj = mode == MODE_XADJ;
        switch (p.Nint[0]) {
            case 64: return adj ? v2::adj_x_launch<T, 64>(a, grid, s) : v2::x2_launch<T, 64>(a, mode, grid, s);
            case 128: return adj ? v2::adj_x_launch<T, 128>(a, grid, s) : v2::x2_launch<T, 128>(a, mode, grid, s);
            case 256: return adj ? v2::adj_x_launch<T, 256>(a, grid, s) : v2::x2_launch<T, 256>(a, mode, grid, s);
            case 512: return adj ? v2::adj_x_launch<T, 512>(a, grid, s) : v2::x2_launch<T, 512>(a, mode, grid, s);
            case 96: return adj ? v2::adj_x_launch<T, 96>(a, grid, s) : v2::x2_launch<T, 96>(a, mode, grid, s);
            case 200: return adj ? v2::adj_x_launch<T, 200>(a, grid, s) : v2::x2_launch<T, 200>(a, mode, grid, s);
            case 384: return adj ? v2::adj_x_launch<T, 384>(a, grid, s) : v2::x2_launch<T, 384>(a, mode, grid, s);
            default: return adj ? v2::adj_x_launch<T, 1024>(a, grid, s) : v2::x2_launch<T, 1024>(a, mode, grid, s);
        }
    }
    if (mode == MODE_XADJ) return cudaErrorNotSupported;
    return dispatch_x<T>(p, a, mode, grid, tile_smem<T>(p, 0), s);
}

template <typename T>
static cudaError_t run_x(const Plan& p, int mode, const Arr<T>& in, const Arr<T>& out, int out_fill,
                         double stage_frac, cudaStream_t s) {
    dim3 grid;
    const XArgs<T> a = x_args<T>(p, in, out, out_fill, stage_frac, grid);
    return launch_x<T>(p, mode, a, grid, s);
}

// ---- 1D: the spectral combination as a pointwise pass ------------------------------------
//
// With one axis the transform of the x pass is the whole transform: after the x pass (T, f, T)
// the work array holds F(f) in spectral space, and the stage combination (Algorithm 1) is pointwise;
// its result times 1/C is what the next x pass transforms back.  mode T0 (load): U <- W, W <- W/C;
// TA/TB/TC/TD as in the slow-axis passes with F = W.
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) combine1d_kernel(const ColArgs<T> a, long long total, long long plane) {
    const T invC = (T)a.invC, tau = (T)a.tau;
    T* W = const_cast<T*>(a.in);
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(e / plane);                 // species
        const T F = W[e];
        T Q = 0, ph = 0, R = 0, p1 = 0, p2 = 0, p3 = 0;
        if (MODE != MODE_T0) {
            if (a.CL) {
                const T L = (T)a.cl_mult[h] * a.CL[h ? e - plane + a.clB : e];
                if (MODE == MODE_TD) p13_rphi<T>(L, tau, R, p1, p2, p3);
                else p13_qphi<T>(L, tau, Q, ph);
            } else if (MODE == MODE_TD) {
                R = a.CR[4 * e]; p1 = a.CR[4 * e + 1]; p2 = a.CR[4 * e + 2]; p3 = a.CR[4 * e + 3];
            } else {
                Q = a.CQ[2 * e]; ph = a.CQ[2 * e + 1];
            }
        }
        T out;
        if (MODE == MODE_T0) {
            a.U[e] = F;
            out = F;
        } else if (MODE == MODE_TA || MODE == MODE_TB) {
            if (MODE == MODE_TA) a.F1[e] = F; else a.F2[e] = F;
            out = Q * a.U[e] + ph * F;
        } else if (MODE == MODE_TC) {
            a.F3[e] = F;
            const T f1 = a.F1[e];
            const T ah = Q * a.U[e] + ph * f1;
            out = Q * ah + ph * ((T)2 * F - f1);
        } else {
            const T un = R * a.U[e] + p1 * a.F1[e] + p2 * (a.F2[e] + a.F3[e]) + p3 * F;
            if (a.F4) a.F4[e] = F;
            a.U[e] = un;
            out = un;
        }
        W[e] = out * invC;
    }
    if (MODE == MODE_TD && blockIdx.x == 0 && threadIdx.x == 0) a.clock->k += 1;
}

template <typename T>
static cudaError_t run_combine1d(const Plan& p, int mode, const Arr<T>& W, cudaStream_t s,
                                 const StepSave* sv = nullptr) {
    dim3 grid;
    ColArgs<T> a = col_args<T>(p, 0, W, W, 1.0, grid);
    if (sv) {   // the stage spectra of this step go to the recomputation arrays
        a.F1 = static_cast<T*>(sv->F[0]);
        a.F2 = static_cast<T*>(sv->F[1]);
        a.F3 = static_cast<T*>(sv->F[2]);
        a.F4 = static_cast<T*>(sv->F[3]);
    }
    const long long total = (long long)p.S * p.plane;
    const int blocks = (int)((total + kThreads - 1) / kThreads < 1024 ? (total + kThreads - 1) / kThreads : 1024);
    switch (mode) {
        case MODE_T0: combine1d_kernel<T, MODE_T0><<<blocks, kThreads, 0, s>>>(a, total, p.plane); break;
        case MODE_TA: combine1d_kernel<T, MODE_TA><<<blocks, kThreads, 0, s>>>(a, total, p.plane); break;
        case MODE_TB: combine1d_kernel<T, MODE_TB><<<blocks, kThreads, 0, s>>>(a, total, p.plane); break;
        case MODE_TC: combine1d_kernel<T, MODE_TC><<<blocks, kThreads, 0, s>>>(a, total, p.plane); break;
        default: combine1d_kernel<T, MODE_TD><<<blocks, kThreads, 0, s>>>(a, total, p.plane); break;
    }
    return cudaGetLastError();
}

// Reverse of the 1D stage combinations (the adjoint's slow-axis modes without the slow-axis
// transform: in 1D the combination acts on the x spectra directly).  Element e of [S][pitch], mode
// index kx = e mod pitch; tilde cotangents as in the multi-dimensional sweep, t = in * (1/C):
//   ENTRY: out = phi3 Ub                               (cotangents of R13, phi1, phi2, phi3)
//   CB:    Cb = t;  out = phi2 Ub + 2 phi Cb
//   BA:    Bb = t;  out = phi2 Ub + phi Bb
//   AU:    Ab = Q Cb + t;  out = phi1 Ub - phi Cb + phi Ab
//   EXIT:  Ub <- R13 Ub + Q (Bb + Ab) + t
template <typename T, int MODE>
__global__ void __launch_bounds__(kThreads) adj_combine1d_kernel(const ColArgs<T> a, long long total, long long plane,
                                                                  int pitch) {
    const bool neu = a.ax.bc == SFRD_BC_NEUMANN;
    const T invC = (T)a.invC;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int h = (int)(e / plane);
        const int kx = (int)(e % plane) % pitch;
        if (kx >= a.nk[0]) continue;                      // padding: zeros in and out
        const double w = v2::endw(kx, a.nk[0], neu);
        const int s = a.S == 2 ? h : 0;
        const T ub = a.Ub[e];
        double cb[6] = {0, 0, 0, 0, 0, 0};
        if (MODE == MODE_ADJ_ENTRY) {
            const double wu = w * (double)ub;
            cb[0] = wu * a.U[e];
            cb[3] = wu * a.F1[e];
            cb[4] = wu * ((double)a.F2[e] + a.F3[e]);
            cb[5] = wu * a.F4[e];
            a.out[e] = a.CR[4 * e + 3] * ub;
        } else {
            const T t = a.in[e] * invC;
            const T Q = a.CQ[2 * e], ph = a.CQ[2 * e + 1];
            if (MODE == MODE_ADJ_CB) {
                a.Cb[e] = t;
                cb[1] = w * (double)t * ((double)Q * a.U[e] + (double)ph * a.F1[e]);
                cb[2] = w * (double)t * (2.0 * a.F3[e] - a.F1[e]);
                a.out[e] = a.CR[4 * e + 2] * ub + (T)2 * ph * t;
            } else if (MODE == MODE_ADJ_BA) {
                a.Bb[e] = t;
                cb[1] = w * (double)t * a.U[e];
                cb[2] = w * (double)t * a.F2[e];
                a.out[e] = a.CR[4 * e + 2] * ub + ph * t;
            } else if (MODE == MODE_ADJ_AU) {
                const T cbv = a.Cb[e];
                const T ah = Q * cbv + t;
                a.Ab[e] = ah;
                cb[1] = w * (double)ah * a.U[e];
                cb[2] = w * (double)ah * a.F1[e];
                a.out[e] = a.CR[4 * e + 1] * ub - ph * cbv + ph * ah;
            } else {
                a.Ub[e] = a.CR[4 * e] * ub + Q * (a.Bb[e] + a.Ab[e]) + t;
            }
        }
        if (MODE != MODE_ADJ_EXIT) v2::coef_grad(a, s, kx, 0, 0, cb, acc);
    }
    v2::flush_sums<4>(acc, a.grad);
}

// One reverse 1D combination: in -> out (may alias: every element is read before it is written).
template <typename T>
static cudaError_t run_adj_combine1d(const Plan& p, int mode, ColArgs<T> a, const T* in, T* out, cudaStream_t s) {
    a.in = in;
    a.out = out;
    const long long total = (long long)p.S * p.plane;
    const int blocks = (int)((total + kThreads - 1) / kThreads < 1024 ? (total + kThreads - 1) / kThreads : 1024);
    const int pitch = (int)p.pitch;
    switch (mode) {
        case MODE_ADJ_ENTRY: adj_combine1d_kernel<T, MODE_ADJ_ENTRY><<<blocks, kThreads, 0, s>>>(a, total, p.plane, pitch); break;
        case MODE_ADJ_CB: adj_combine1d_kernel<T, MODE_ADJ_CB><<<blocks, kThreads, 0, s>>>(a, total, p.plane, pitch); break;
        case MODE_ADJ_BA: adj_combine1d_kernel<T, MODE_ADJ_BA><<<blocks, kThreads, 0, s>>>(a, total, p.plane, pitch); break;
        case MODE_ADJ_AU: adj_combine1d_kernel<T, MODE_ADJ_AU><<<blocks, kThreads, 0, s>>>(a, total, p.plane, pitch); break;
        default: adj_combine1d_kernel<T, MODE_ADJ_EXIT><<<blocks, kThreads, 0, s>>>(a, total, p.plane, pitch); break;
    }
    return cudaGetLastError();
}

// out (internal layout) = scale * in (dense [S][n]) for the 1D inverse transform entry point.
template <typename T>
__global__ void scale1d_kernel(const T* __restrict__ in, T* __restrict__ out, int n, int pitch, int S, double scale) {
    const long long total = (long long)S * pitch;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e % pitch), sp = (int)(e / pitch);
        out[e] = x < n ? (T)scale * in[(long long)sp * n + x] : (T)0;
    }
}

// One step.  With `ev` non-null, event ev[i] is recorded before launch i and
// ev[i+1] after it, and kind[i] receives the pass kind (PassKind).  With `sv`
// non-null the stage spectra and physical stage values are written to the
// arrays it names (checkpointed recomputation for the adjoint).
template <typename T>
static cudaError_t step_impl(Plan& p, cudaStream_t s, cudaEvent_t* ev, int* kind, int cap,
                             const StepSave* sv = nullptr) {
    const Arr<T> W = internal_arr<T>(p, p.off_W);
    const int slow = p.dim == 3 ? 2 : 1;
    static const double frac[4] = {0.0, 0.5, 0.5, 1.0};
    int i = 0;
    auto mark = [&](int k) -> cudaError_t {
        if (!ev || i >= cap) return cudaSuccess;
        if (kind) kind[i] = k;
        return cudaEventRecord(ev[i], s);
    };
    auto done = [&]() -> cudaError_t {
        cudaError_t e = cudaSuccess;
        if (ev && i < cap) e = cudaEventRecord(ev[i + 1], s);
        ++i;
        return e;
    };
    for (int st = 0; st < 4; ++st) {
        if (p.dim == 1) {
            SFRD_TRY(mark(PASS_X));
            {
                dim3 grid;
                XArgs<T> a = x_args<T>(p, W, W, p.pitch, frac[st], grid);
                if (sv) a.save = static_cast<T*>(sv->stage[st]);
                SFRD_TRY(launch_x<T>(p, MODE_REACT, a, grid, s));
            }
            SFRD_TRY(done());
            SFRD_TRY(mark(PASS_SLOW_A + st));
            SFRD_TRY(run_combine1d<T>(p, MODE_TA + st, W, s, sv));
            SFRD_TRY(done());
            continue;
        }
        if (p.dim == 3) {
            SFRD_TRY(mark(PASS_MID));
            SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W, W, 1.0, s));
            SFRD_TRY(done());
        }
        SFRD_TRY(mark(PASS_X));
        {
            dim3 grid;
            XArgs<T> a = x_args<T>(p, W, W, p.pitch, frac[st], grid);
            if (sv) a.save = static_cast<T*>(sv->stage[st]);
            SFRD_TRY(launch_x<T>(p, MODE_REACT, a, grid, s));
        }
        SFRD_TRY(done());
        if (p.dim == 3) {
            SFRD_TRY(mark(PASS_MID));
            SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W, W, 1.0, s));
            SFRD_TRY(done());
        }
        SFRD_TRY(mark(PASS_SLOW_A + st));
        {
            dim3 grid;
            ColArgs<T> a = col_args<T>(p, slow, W, W, 1.0, grid, true);
            if (sv) {
                a.F1 = static_cast<T*>(sv->F[0]);
                a.F2 = static_cast<T*>(sv->F[1]);
                a.F3 = static_cast<T*>(sv->F[2]);
                a.F4 = static_cast<T*>(sv->F[3]);
            }
            SFRD_TRY(launch_col<T>(p, slow, MODE_TA + st, a, grid, s));
        }
        SFRD_TRY(done());
    }
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_step(Plan& p, cudaStream_t s) {
    return step_impl<T>(p, s, nullptr, nullptr, 0);
}

template <typename T>
cudaError_t launch_step_profiled(Plan& p, cudaStream_t s, cudaEvent_t* ev, int* kind, int cap) {
    return step_impl<T>(p, s, ev, kind, cap);
}

template <typename T>
cudaError_t launch_load(Plan& p, const void* u0, cudaStream_t s) {
    const Arr<T> W = internal_arr<T>(p, p.off_W);
    const int slow = p.dim == 3 ? 2 : 1;
    SFRD_TRY(run_x<T>(p, MODE_PLAIN, dense_arr<T>(p, u0), W, p.pitch, 0.0, s));
    if (p.dim == 1) return run_combine1d<T>(p, MODE_T0, W, s);
    if (p.dim == 3) SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W, W, 1.0, s));
    return run_col<T>(p, slow, MODE_T0, W, W, 1.0, s);
}

template <typename T>
cudaError_t launch_store(Plan& p, void* u, cudaStream_t s) {
    const Arr<T> W = internal_arr<T>(p, p.off_W);
    const Arr<T> W2 = internal_arr<T>(p, p.off_W2);
    if (p.dim == 3) {
        SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W, W2, 1.0, s));
        return run_x<T>(p, MODE_PLAIN, W2, dense_arr<T>(p, u), 0, 0.0, s);
    }
    return run_x<T>(p, MODE_PLAIN, W, dense_arr<T>(p, u), 0, 0.0, s);
}

template <typename T>
cudaError_t launch_forward(Plan& p, const void* u, void* uhat, cudaStream_t s) {
    const Arr<T> W2 = internal_arr<T>(p, p.off_W2);
    const int slow = p.dim == 3 ? 2 : 1;
    if (p.dim == 1) return run_x<T>(p, MODE_PLAIN, dense_arr<T>(p, u), dense_arr<T>(p, uhat), 0, 0.0, s);
    SFRD_TRY(run_x<T>(p, MODE_PLAIN, dense_arr<T>(p, u), W2, p.pitch, 0.0, s));
    if (p.dim == 3) SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W2, W2, 1.0, s));
    return run_col<T>(p, slow, MODE_PLAIN, W2, dense_arr<T>(p, uhat), 1.0, s);
}

template <typename T>
cudaError_t launch_inverse(Plan& p, const void* uhat, void* u, cudaStream_t s) {
    const Arr<T> W2 = internal_arr<T>(p, p.off_W2);
    const int slow = p.dim == 3 ? 2 : 1;
    double C = 1.0;
    for (int k = 0; k < p.dim; ++k) C *= (p.bc == SFRD_BC_PERIODIC) ? (double)p.Nint[k] : 0.5 * (double)p.Nint[k];
    SFRD_TRY(cudaMemsetAsync(p.ws + p.off_W2, 0, (size_t)p.S * p.plane * sizeof(T), s));
    if (p.dim == 1) {
        scale1d_kernel<T><<<64, kThreads, 0, s>>>(static_cast<const T*>(uhat), wsT<T>(p, p.off_W2), p.n[0], p.pitch,
                                                   p.S, 1.0 / C);
        SFRD_TRY(cudaGetLastError());
        return run_x<T>(p, MODE_PLAIN, W2, dense_arr<T>(p, u), 0, 0.0, s);
    }
    SFRD_TRY(run_col<T>(p, slow, MODE_PLAIN, dense_arr<T>(p, uhat), W2, 1.0 / C, s));
    if (p.dim == 3) SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W2, W2, 1.0, s));
    return run_x<T>(p, MODE_PLAIN, W2, dense_arr<T>(p, u), 0, 0.0, s);
}

// Sets *flag when any value of the resident spectral state is not finite (the flag is cleared by the
// caller first).  A spectral value is finite exactly when the run has not blown up or been fed a
// non-finite field: every transform mixes all values of a line.
template <typename T>
__global__ void finite_check_kernel(const T* __restrict__ x, long long n, int* flag) {
    int bad = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) *flag = 1;
}

template <typename T>
cudaError_t launch_finite_check(Plan& p, cudaStream_t s) {
    int* flag = reinterpret_cast<int*>(p.ws + p.off_flag);
    SFRD_TRY(cudaMemsetAsync(flag, 0, sizeof(int), s));
    finite_check_kernel<T><<<304, kThreads, 0, s>>>(wsT<T>(p, p.off_U), (long long)p.S * p.plane, flag);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coef_init(Plan& p, cudaStream_t s) {
    const double* lx = reinterpret_cast<const double*>(p.ws + p.off_lam[0]);
    const double* ly = reinterpret_cast<const double*>(p.ws + p.off_lam[1]);
    const double* lz = reinterpret_cast<const double*>(p.ws + p.off_lam[2]);
    const double a1 = p.S == 2 ? p.alpha[1] : p.alpha[0];
    const double k1 = p.S == 2 ? p.kappa[1] : p.kappa[0];
    if (p.coef_mode == SFRD_COEF_RATIONAL)
        coef_l_kernel<T><<<1024, 256, 0, s>>>(lx, ly, lz, p.n[0], p.n[1], p.n[2], p.pitch, p.cl_shared ? 1 : p.S,
                                              p.cl_shared, p.alpha[0], a1, p.kappa[0], k1, p.dt,
                                              wsT<T>(p, p.off_CL));
    else
        coef_init_kernel<T><<<1024, 256, 0, s>>>(lx, ly, lz, p.n[0], p.n[1], p.n[2], p.pitch, p.S, p.alpha[0], a1,
                                                 p.kappa[0], k1, p.dt, p.scheme, wsT<T>(p, p.off_CQ),
                                                 wsT<T>(p, p.off_CR));
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coef_copy(Plan& p, int which, void* out, cudaStream_t s) {
    if (p.coef_mode == SFRD_COEF_RATIONAL) {
        const double k1 = p.S == 2 ? p.kappa[1] : p.kappa[0];
        coef_eval_kernel<T><<<1024, 256, 0, s>>>(wsT<T>(p, p.off_CL), p.cl_shared, p.kappa[0], k1, p.dt, which, p.n[0],
                                                 p.n[1], p.n[2], p.pitch, p.S, static_cast<T*>(out));
        return cudaGetLastError();
    }
    coef_copy_kernel<T><<<1024, 256, 0, s>>>(wsT<T>(p, p.off_CQ), wsT<T>(p, p.off_CR), which, p.n[0], p.n[1], p.n[2],
                                             p.pitch, p.S, static_cast<T*>(out));
    return cudaGetLastError();
}

// ---- checkpointed forward and discrete adjoint (register engine) ----------------------

// out = in * w (mul) or in / w (div) with w the product of the Neumann endpoint weights
// (1/2 at nodes 0 and N of each axis) of a dense [S][n_z][n_y][n_x] field.
template <typename T>
__global__ void endpoint_weight_kernel(const T* __restrict__ in, T* __restrict__ out, int nx, int ny, int nz, int S,
                                       int divide) {
    const long long total = (long long)S * nz * ny * nx;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(idx % nx);
        const long long r = idx / nx;
        const int y = (int)(r % ny);
        const int z = (int)((r / ny) % nz);
        double w = 1.0;
        if (nx > 1 && (x == 0 || x == nx - 1)) w *= 0.5;
        if (ny > 1 && (y == 0 || y == ny - 1)) w *= 0.5;
        if (nz > 1 && (z == 0 || z == nz - 1)) w *= 0.5;
        out[idx] = divide ? (T)(in[idx] / w) : (T)(in[idx] * w);
    }
}

template <typename T>
static cudaError_t dense_weights(const Plan& p, const void* in, void* out, bool divide, cudaStream_t s) {
    if (p.bc != SFRD_BC_NEUMANN) {
        if (in != out) return cudaMemcpyAsync(out, in, (size_t)p.S * p.dense * sizeof(T), cudaMemcpyDeviceToDevice, s);
        return cudaSuccess;
    }
    endpoint_weight_kernel<T><<<512, 256, 0, s>>>(static_cast<const T*>(in), static_cast<T*>(out), p.n[0], p.n[1],
                                                  p.n[2], p.S, divide ? 1 : 0);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_run_checkpointed(Plan& p, void* u, double t0, int64_t nsteps, int64_t K, char* aws,
                                    const AdjLayout& L, cudaStream_t s) {
    SFRD_TRY(launch_set_clock(p, t0, s, 0));
    SFRD_TRY(launch_load<T>(p, u, s));
    for (int64_t seg = 0; seg < L.nseg; ++seg) {
        SFRD_TRY(cudaMemcpyAsync(aws + L.off_ckpt + seg * L.fld, p.ws + p.off_U, L.fld, cudaMemcpyDeviceToDevice, s));
        const int64_t ns = (seg + 1) * K <= nsteps ? K : nsteps - seg * K;
        for (int64_t j = 0; j < ns; ++j) SFRD_TRY(launch_step<T>(p, s));
    }
    return launch_store<T>(p, u, s);
}

template <typename T>
cudaError_t launch_adjoint(Plan& p, double t0, int64_t nsteps, int64_t K, char* aws, const AdjLayout& L,
                           const void* dLduT, void* dLdu0, cudaStream_t s) {
    const Arr<T> W = internal_arr<T>(p, p.off_W);
    const Arr<T> W2 = internal_arr<T>(p, p.off_W2);
    const int slow = p.dim == 3 ? 2 : 1;
    double C = 1.0;
    for (int k = 0; k < p.dim; ++k) C *= (p.bc == SFRD_BC_PERIODIC) ? (double)p.Nint[k] : 0.5 * (double)p.Nint[k];
    T* ub = reinterpret_cast<T*>(aws + L.off_Ub);
    T* cb = reinterpret_cast<T*>(aws + L.off_Cb);
    T* bb = reinterpret_cast<T*>(aws + L.off_Bb);
    T* ab = reinterpret_cast<T*>(aws + L.off_Ab);
    double* grad = reinterpret_cast<double*>(aws + L.off_grad);
    const Arr<T> UB{ub, p.pitch, p.plane, p.pitch};
    const Arr<T> D = dense_arr<T>(p, p.ws + p.off_D);
    SFRD_TRY(cudaMemsetAsync(grad, 0, 16 * sizeof(double), s));
    SFRD_TRY(cudaMemsetAsync(aws + L.off_Ub, 0, 4 * L.fld, s));

    // entry: Ub~ = T(g ./ w) / C
    SFRD_TRY(dense_weights<T>(p, dLduT, p.ws + p.off_D, true, s));
    if (p.dim == 1) {
        scale1d_kernel<T><<<64, kThreads, 0, s>>>(D.ptr, wsT<T>(p, p.off_W2), p.n[0], p.pitch, p.S, 1.0 / C);
        SFRD_TRY(cudaGetLastError());
        SFRD_TRY(run_x<T>(p, MODE_PLAIN, W2, UB, p.pitch, 0.0, s));
    } else {
        SFRD_TRY(run_x<T>(p, MODE_PLAIN, D, W2, p.pitch, 0.0, s));
        if (p.dim == 3) SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W2, W2, 1.0, s));
        SFRD_TRY(run_col<T>(p, slow, MODE_PLAIN, W2, UB, 1.0 / C, s));
    }

    const size_t per_step = 9 * L.fld;   // u^, F1..F4, u, a, b, c
    for (int64_t seg = L.nseg - 1; seg >= 0; --seg) {
        const int64_t k0 = seg * K;
        const int64_t ns = k0 + K <= nsteps ? K : nsteps - k0;
        // recompute the segment from its checkpoint, saving every step's intermediates
        if (p.dim == 1) {   // W = checkpoint, then U = W, W = W / C (the load's last pass)
            SFRD_TRY(cudaMemcpyAsync(p.ws + p.off_W, aws + L.off_ckpt + seg * L.fld, L.fld, cudaMemcpyDeviceToDevice, s));
            SFRD_TRY(run_combine1d<T>(p, MODE_T0, W, s));
        } else {
            SFRD_TRY(cudaMemcpyAsync(p.ws + p.off_U, aws + L.off_ckpt + seg * L.fld, L.fld, cudaMemcpyDeviceToDevice, s));
            SFRD_TRY(run_col<T>(p, slow, MODE_PLAIN, internal_arr<T>(p, p.off_U), W, 1.0 / C, s));
        }
        SFRD_TRY(launch_set_clock(p, t0, s, k0));
        for (int64_t j = 0; j < ns; ++j) {
            char* st = aws + L.off_seg + j * per_step;
            SFRD_TRY(cudaMemcpyAsync(st, p.ws + p.off_U, L.fld, cudaMemcpyDeviceToDevice, s));
            StepSave sv;
            for (int q = 0; q < 4; ++q) {
                sv.F[q] = st + (1 + q) * L.fld;
                sv.stage[q] = st + (5 + q) * L.fld;
            }
            SFRD_TRY(step_impl<T>(p, s, nullptr, nullptr, 0, &sv));
        }
        // reverse sweep over the segment
        for (int64_t j = ns - 1; j >= 0; --j) {
            char* st = aws + L.off_seg + j * per_step;
            auto patch = [&](ColArgs<T>& a) {
                a.U = reinterpret_cast<T*>(st);
                a.F1 = reinterpret_cast<T*>(st + 1 * L.fld);
                a.F2 = reinterpret_cast<T*>(st + 2 * L.fld);
                a.F3 = reinterpret_cast<T*>(st + 3 * L.fld);
                a.F4 = reinterpret_cast<T*>(st + 4 * L.fld);
                a.Ub = ub;
                a.Cb = cb;
                a.Bb = bb;
                a.Ab = ab;
                a.grad = grad;
            };
            auto slow_pass = [&](int mode, const Arr<T>& in) -> cudaError_t {
                dim3 grid;
                if (p.dim == 1) {   // the combination acts on the x spectra directly
                    ColArgs<T> a = col_args<T>(p, 0, in, W, 1.0, grid);
                    patch(a);
                    return run_adj_combine1d<T>(p, mode, a, in.ptr, const_cast<T*>(W.ptr), s);
                }
                ColArgs<T> a = col_args<T>(p, slow, in, W, 1.0, grid);
                patch(a);
                return launch_col<T>(p, slow, mode, a, grid, s);
            };
            auto x_pass = [&](int stage) -> cudaError_t {
                dim3 grid;
                XArgs<T> a = x_args<T>(p, W, W, p.pitch, 0.0, grid);
                a.state = reinterpret_cast<const T*>(st + (5 + stage) * L.fld);
                a.grad = grad;
                return launch_x<T>(p, MODE_XADJ, a, grid, s);
            };
            auto chain = [&](int stage) -> cudaError_t {
                if (p.dim == 3) SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W, W, 1.0, s));
                SFRD_TRY(x_pass(stage));
                if (p.dim == 3) SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W, W, 1.0, s));
                return cudaSuccess;
            };
            SFRD_TRY(slow_pass(MODE_ADJ_ENTRY, UB));
            SFRD_TRY(chain(3));
            SFRD_TRY(slow_pass(MODE_ADJ_CB, W));
            SFRD_TRY(chain(2));
            SFRD_TRY(slow_pass(MODE_ADJ_BA, W));
            SFRD_TRY(chain(1));
            SFRD_TRY(slow_pass(MODE_ADJ_AU, W));
            SFRD_TRY(chain(0));
            SFRD_TRY(slow_pass(MODE_ADJ_EXIT, W));
        }
    }
    // exit: dL/du0 = w .* T(Ub~)
    if (p.dim == 1) {
        SFRD_TRY(run_x<T>(p, MODE_PLAIN, UB, D, 0, 0.0, s));
    } else {
        SFRD_TRY(run_x<T>(p, MODE_PLAIN, UB, W2, p.pitch, 0.0, s));
        if (p.dim == 3) SFRD_TRY(run_col<T>(p, 1, MODE_PLAIN, W2, W2, 1.0, s));
        SFRD_TRY(run_col<T>(p, slow, MODE_PLAIN, W2, D, 1.0, s));
    }
    return dense_weights<T>(p, p.ws + p.off_D, dLdu0, false, s);
}

#define SFRD_INSTANTIATE(T)                                                                  \
    template cudaError_t launch_step<T>(Plan&, cudaStream_t);                                \
    template cudaError_t launch_step_profiled<T>(Plan&, cudaStream_t, cudaEvent_t*, int*, int); \
    template cudaError_t launch_load<T>(Plan&, const void*, cudaStream_t);                   \
    template cudaError_t launch_store<T>(Plan&, void*, cudaStream_t);                        \
    template cudaError_t launch_forward<T>(Plan&, const void*, void*, cudaStream_t);         \
    template cudaError_t launch_inverse<T>(Plan&, const void*, void*, cudaStream_t);         \
    template cudaError_t launch_coef_init<T>(Plan&, cudaStream_t);                           \
    template cudaError_t launch_finite_check<T>(Plan&, cudaStream_t);                        \
    template cudaError_t launch_coef_copy<T>(Plan&, int, void*, cudaStream_t);          \
    template cudaError_t prepare_kernels<T>(const Plan&);                                  \
    template cudaError_t launch_run_checkpointed<T>(Plan&, void*, double, int64_t, int64_t, char*,       \
                                                    const AdjLayout&, cudaStream_t);                      \
    template cudaError_t launch_adjoint<T>(Plan&, double, int64_t, int64_t, char*, const AdjLayout&,     \
                                           const void*, void*, cudaStream_t);

}  // namespace sfrd
