// Discrete adjoint of the ETDRK4-P13 step on the register FFT engine.
//
// The step (Eq. ETDRK4P13 / Algorithm 1, in this library's spectral form with
// F = T, the unnormalised separable real transform, and P = T / C its inverse):
//   u = P(u^); F1 = F f(u); a^ = Q u^ + phi F1; a = P(a^); F2 = F f(a);
//   b^ = Q u^ + phi F2; b = P(b^); F3 = F f(b); c^ = Q a^ + phi (2 F3 - F1);
//   c = P(c^); F4 = F f(c); u^' = R u^ + phi1 F1 + phi2 (F2 + F3) + phi3 F4.
// Its reverse sweep needs the transposes F^T = T^T and P^T = T^T / C.  T is
// symmetric for the Hartley and sine transforms; for the weighted DCT-I,
// T^T = W T W^{-1} with W = diag of the endpoint weights (1/2 at nodes 0 and N
// of every axis).  Every other operation of the step is diagonal in space or in
// mode index, so it commutes with W, and the whole reverse sweep equals
// W [the same sweep with T in place of T^T] W^{-1}.  The kernels therefore run
// that sweep on "tilde" cotangents y~ = W^{-1} y with plain T, and apply W only
// where a cotangent meets a primal value: the coefficient cotangents
// (w_k y~_k x_k), the reaction-parameter sums (w(x) ...), and the two ends.
//
// Reverse of one step, on tilde spectra (Ub = d l / d u^', updated in place):
//   c-chain:  F4b = phi3 Ub  -> T -> J_f(c)^T -> T/C -> Cb
//   b-chain:  F3b = phi2 Ub + 2 phi Cb -> T -> J_f(b)^T -> T/C -> Bb
//   a-chain:  F2b = phi2 Ub + phi Bb   -> T -> J_f(a)^T -> T/C (+ Q Cb) -> Ab
//   u-chain:  F1b = phi1 Ub - phi Cb + phi Ab -> T -> J_f(u)^T -> T/C
//             Ub <- R Ub + Q Bb + Q Ab + (that)
// and the coefficient cotangents R: Ub u^, phi1: Ub F1, phi2: Ub (F2 + F3),
// phi3: Ub F4, Q: Cb a^ + Bb u^ + Ab u^, phi: Cb (2F3 - F1) + Bb F2 + Ab F1,
// which reach kappa_s and alpha_s through L = kappa_s tau Lambda^{alpha_s/2}.
#pragma once

#include "adjgrad.cuh"
#include "passes2.cuh"

namespace sfrd {
namespace v2 {

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(kThreads, (min_blocks<T, N, MODE_TA>())) adj_col_kernel(const ColArgs<T> a) {
    constexpr int CC = TileOf<T, N>::CC;
    using E = typename TileOf<T, N>::E;
    using C = typename E::C;
    constexpr int LD = E::LD, G = E::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* red = buf + E::ROWS * LD;
    C* red2 = red + G * CC;
    C* tws = red2 + G * CC;
    const int tid = threadIdx.x, c = tid % CC, g = tid / CC;
    const AxisDev& ax = a.ax;
    const int n = ax.n, bc = ax.bc;
    const bool neu = bc == SFRD_BC_NEUMANN;
    const C* tw = static_cast<const C*>(ax.tw);
    const int twstride = bc == SFRD_BC_PERIODIC ? 1 : 2;
    for (int i = tid; i < N * twstride; i += kThreads) tws[i] = __ldg(tw + i);
    const int xA = blockIdx.x * a.xw + c * a.cstride, xB = xA + a.bshift;
    const int other = blockIdx.y;
    const bool okA = xA < a.in_xlim, okB = xB < a.in_xlim;
    const long long base = (long long)other * a.in_sOther + xA;
    const T invC = (T)a.invC;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};

    // mode indices (kx, ky, kz) and spectral weight of element k (along the slow axis) of column h
    // (padding columns x >= n_x carry zeros and report kx = -1: no coefficient gradient there)
    auto mode_of = [&](int k, int h, int& s, int& kx, int& ky, int& kz) -> double {
        const int x = h ? xB : xA;
        s = (a.S == 2) ? h : 0;
        kx = x < a.nk[0] ? x : -1;
        if (a.dim == 3) { ky = other; kz = k; } else { ky = k; kz = 0; }
        return kx < 0 ? 0.0 : endw(kx, a.nk[0], neu) * endw(ky, a.nk[1], neu) * endw(kz, a.nk[2], neu);
    };

    if (MODE == MODE_ADJ_ENTRY) {
        // F4b = phi3 Ub; cotangents of R13, phi1, phi2, phi3
        for (int i = g; i < n; i += G) {
            C z;
            T zz[2] = {0, 0};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h ? okB : okA)) continue;
                const long long e = base + (long long)i * a.in_sAxis + (h ? a.in_offB : 0);
                const T ub = a.Ub[e];
                zz[h] = a.CR[4 * e + 3] * ub;
                int s, kx, ky, kz;
                const double w = mode_of(i, h, s, kx, ky, kz) * (double)ub;
                const double cb[6] = {w * a.U[e], 0.0, 0.0, w * a.F1[e], w * ((double)a.F2[e] + a.F3[e]),
                                      w * a.F4[e]};
                if (kx >= 0) coef_grad(a, s, kx, ky, kz, cb, acc);
            }
            z.x = zz[0];
            z.y = zz[1];
            buf[i * LD + c] = z;
        }
    } else {
        const T* pA = a.in + base;
        for (int i = g; i < n; i += G) {
            C z;
            z.x = okA ? pA[(long long)i * a.in_sAxis] : (T)0;
            z.y = okB ? pA[(long long)i * a.in_sAxis + a.in_offB] : (T)0;
            buf[i * LD + c] = z;
        }
    }
    __syncthreads();
    E::forward(buf, red2, bc, tws, twstride, c, g);

    if (MODE != MODE_ADJ_ENTRY) {
        E::post(buf, red, red2, bc, c, g, [&](int k, C v) {
            T sv[2] = {0, 0};
            const T vv[2] = {v.x, v.y};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!(h ? okB : okA)) continue;
                const long long e = base + (long long)k * a.in_sAxis + (h ? a.in_offB : 0);
                const T t = vv[h] * invC;
                const T Q = a.CQ[2 * e], ph = a.CQ[2 * e + 1];
                const T ub = a.Ub[e];
                int s, kx, ky, kz;
                const double w = mode_of(k, h, s, kx, ky, kz);
                double cb[6] = {0, 0, 0, 0, 0, 0};
                if (MODE == MODE_ADJ_CB) {
                    a.Cb[e] = t;
                    const T u = a.U[e], f1 = a.F1[e], f3 = a.F3[e];
                    cb[1] = w * (double)t * ((double)Q * u + (double)ph * f1);
                    cb[2] = w * (double)t * (2.0 * f3 - f1);
                    sv[h] = a.CR[4 * e + 2] * ub + (T)2 * ph * t;
                } else if (MODE == MODE_ADJ_BA) {
                    a.Bb[e] = t;
                    cb[1] = w * (double)t * a.U[e];
                    cb[2] = w * (double)t * a.F2[e];
                    sv[h] = a.CR[4 * e + 2] * ub + ph * t;
                } else if (MODE == MODE_ADJ_AU) {
                    const T cbv = a.Cb[e];
                    const T ah = Q * cbv + t;
                    a.Ab[e] = ah;
                    cb[1] = w * (double)ah * a.U[e];
                    cb[2] = w * (double)ah * a.F1[e];
                    sv[h] = a.CR[4 * e + 1] * ub - ph * cbv + ph * ah;
                } else {  // MODE_ADJ_EXIT
                    a.Ub[e] = a.CR[4 * e] * ub + Q * (a.Bb[e] + a.Ab[e]) + t;
                }
                if (MODE != MODE_ADJ_EXIT && kx >= 0) coef_grad(a, s, kx, ky, kz, cb, acc);
            }
            if (MODE != MODE_ADJ_EXIT) {
                C z;
                z.x = sv[0];
                z.y = sv[1];
                buf[k * LD + c] = z;
            }
        });
    }
    if (MODE != MODE_ADJ_EXIT) {
        if (MODE != MODE_ADJ_ENTRY) {
            __syncthreads();
            E::forward(buf, red2, bc, tws, twstride, c, g);
        }
        const bool oA = xA < a.out_xlim, oB = xB < a.out_xlim;
        T* qA = a.out + (long long)other * a.out_sOther + xA;
        E::post(buf, red, red2, bc, c, g, [&](int i, C v) {
            if (oA) qA[(long long)i * a.out_sAxis] = v.x;
            if (oB) qA[(long long)i * a.out_sAxis + a.out_offB] = v.y;
        });
    }
    flush_sums<4>(acc, a.grad);
}

// Contiguous axis: out = T(J_f(state)^T T(in)), dL/dparams += sum_x w(x) (df/dp) . T(in).
template <typename T, int N>
__global__ void __launch_bounds__(kThreads, (min_blocks<T, N, MODE_TA>())) adj_x_kernel(const XArgs<T> a) {
    constexpr int CC = TileOf<T, N>::CC;
    using E = typename TileOf<T, N>::E;
    using C = typename E::C;
    constexpr int LD = E::LD, G = E::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* red = buf + E::ROWS * LD;
    C* red2 = red + G * CC;
    C* tws = red2 + G * CC;
    const int tid = threadIdx.x, c = tid % CC, g = tid / CC;
    const AxisDev& ax = a.ax;
    const int n = ax.n, bc = ax.bc;
    const bool neu = bc == SFRD_BC_NEUMANN;
    const C* tw = static_cast<const C*>(ax.tw);
    const int twstride = bc == SFRD_BC_PERIODIC ? 1 : 2;
    for (int i = tid; i < N * twstride; i += kThreads) tws[i] = __ldg(tw + i);
    const int shiftB = (a.S == 2) ? 0 : CC;
    const int r0 = blockIdx.x * (a.S == 2 ? CC : 2 * CC);
    constexpr int NW = kThreads / 32, RW = (CC + NW - 1) / NW;
    const int w = tid >> 5, l = tid & 31;
    double dp[5] = {0, 0, 0, 0, 0};

    for (int rr = 0; rr < RW; ++rr) {
        const int cc = w + rr * NW;
        if (cc >= CC) continue;
        const int rA = r0 + cc, rB = rA + shiftB;
        const T* pA = a.in + (long long)rA * a.in_pitch;
        for (int x = l; x < n; x += 32) {
            C z;
            z.x = rA < a.rows ? pA[x] : (T)0;
            z.y = rB < a.rows ? pA[a.in_offB + x] : (T)0;
            buf[x * LD + cc] = z;
        }
    }
    __syncthreads();
    E::forward(buf, red2, bc, tws, twstride, c, g);
    E::post(buf, red, red2, bc, c, g, [&](int i, C v) { buf[i * LD + c] = v; });
    __syncthreads();
    for (int rr = 0; rr < RW; ++rr) {
        const int cc = w + rr * NW;
        if (cc >= CC) continue;
        const int rA = r0 + cc, rB = rA + shiftB;
        const T* st = a.state + (long long)rA * a.in_pitch;
        const int yA = rA % a.ny, zA = rA / a.ny, yB = rB % a.ny, zB = rB / a.ny;
        const double wA = endw(yA, a.ny, neu) * endw(zA, a.nz, neu);
        const double wB = endw(yB, a.ny, neu) * endw(zB, a.nz, neu);
        for (int x = l; x < n; x += 32) {
            const C y = buf[x * LD + cc];
            const double wx = endw(x, n, neu);
            C gv;
            if (a.S == 2) {
                const T u = rA < a.rows ? st[x] : (T)0, vv = rA < a.rows ? st[a.in_offB + x] : (T)0;
                react2_vjp<T>(a.re, u, vv, y.x, y.y, gv.x, gv.y, (rA < a.rows) ? wx * wA : 0.0, dp);
            } else {
                const T uA = rA < a.rows ? st[x] : (T)0, uB = rB < a.rows ? st[a.in_offB + x] : (T)0;
                gv.x = react1_vjp<T>(a.re, uA, y.x, (rA < a.rows) ? wx * wA : 0.0, dp);
                gv.y = react1_vjp<T>(a.re, uB, y.y, (rB < a.rows) ? wx * wB : 0.0, dp);
            }
            buf[x * LD + cc] = gv;
        }
    }
    __syncthreads();
    E::forward(buf, red2, bc, tws, twstride, c, g);
    E::post(buf, red, red2, bc, c, g, [&](int i, C v) { buf[i * LD + c] = v; });
    __syncthreads();
    for (int rr = 0; rr < RW; ++rr) {
        const int cc = w + rr * NW;
        if (cc >= CC) continue;
        const int rA = r0 + cc, rB = rA + shiftB;
        T* qA = a.out + (long long)rA * a.out_pitch;
        const int xend = a.out_fill > n ? a.out_fill : n;
        for (int x = l; x < xend; x += 32) {
            const C v = x < n ? buf[x * LD + cc] : czero<C>();
            if (rA < a.rows) qA[x] = v.x;
            if (rB < a.rows) qA[a.out_offB + x] = v.y;
        }
    }
    flush_sums<5>(dp, a.grad + 4);
}

template <typename T, int N>
cudaError_t adj_col_launch(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    const size_t smem = TileOf<T, N>::E::smem_bytes();
    void (*k)(const ColArgs<T>) = nullptr;
    switch (mode) {
        case MODE_ADJ_ENTRY: k = adj_col_kernel<T, N, MODE_ADJ_ENTRY>; break;
        case MODE_ADJ_CB: k = adj_col_kernel<T, N, MODE_ADJ_CB>; break;
        case MODE_ADJ_BA: k = adj_col_kernel<T, N, MODE_ADJ_BA>; break;
        case MODE_ADJ_AU: k = adj_col_kernel<T, N, MODE_ADJ_AU>; break;
        default: k = adj_col_kernel<T, N, MODE_ADJ_EXIT>; break;
    }
    k<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t adj_x_launch(const XArgs<T>& a, dim3 grid, cudaStream_t s) {
    adj_x_kernel<T, N><<<grid, kThreads, TileOf<T, N>::E::smem_bytes(), s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t prepare_adj() {
    const int m = kMaxDynSmem2;
    void (*ks[])(const ColArgs<T>) = {adj_col_kernel<T, N, MODE_ADJ_ENTRY>, adj_col_kernel<T, N, MODE_ADJ_CB>,
                                      adj_col_kernel<T, N, MODE_ADJ_BA>, adj_col_kernel<T, N, MODE_ADJ_AU>,
                                      adj_col_kernel<T, N, MODE_ADJ_EXIT>};
    for (auto k : ks) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
        if (e != cudaSuccess) return e;
    }
    return cudaFuncSetAttribute(adj_x_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, m);
}

#define SFRD_ADJ_INSTANTIATE(T, N)                                                               \
    template cudaError_t adj_col_launch<T, N>(const ColArgs<T>&, int, dim3, cudaStream_t);      \
    template cudaError_t adj_x_launch<T, N>(const XArgs<T>&, dim3, cudaStream_t);               \
    template cudaError_t prepare_adj<T, N>();

}  // namespace v2
}  // namespace sfrd
