// Gradient pieces shared by the adjoint passes of every dimension: the endpoint weights of the
// weighted DCT-I, dC/dL of the six coefficient arrays (Pade-(1,3) and Cox-Matthews), their chain to
// dl/dkappa_s and dl/dalpha_s through L = kappa_s tau Lambda^{alpha_s/2}, and warp-level
// accumulation of the sums.
#pragma once

#include "coef.cuh"
#include "sfrd_internal.h"

namespace sfrd {
namespace v2 {

// Endpoint weight of the weighted DCT-I along one axis of n > 1 unknowns.
__device__ __forceinline__ double endw(int k, int n, bool neu) {
    return (neu && n > 1 && (k == 0 || k == n - 1)) ? 0.5 : 1.0;
}

// dC/dL of Algorithm 1's rationals, order R13, Q13, phi, phi1, phi2, phi3 (quotient rule).
__device__ __forceinline__ void dcoef_dL(double L, double tau, double* d) {
    const double D1 = 24.0 + L * (18.0 + L * (6.0 + L)), D2 = 192.0 + L * (72.0 + L * (12.0 + L));
    const double dD1 = 18.0 + L * (12.0 + 3.0 * L), dD2 = 72.0 + L * (24.0 + 3.0 * L);
    const double i1 = 1.0 / (D1 * D1), i2 = 1.0 / (D2 * D2);
    d[0] = (-6.0 * D1 - (24.0 - 6.0 * L) * dD1) * i1;
    d[1] = (-24.0 * D2 - 24.0 * (8.0 - L) * dD2) * i2;
    d[2] = tau * ((12.0 + 2.0 * L) * D2 - (96.0 + L * (12.0 + L)) * dD2) * i2;
    d[3] = tau * (-1.0 * D1 - (4.0 - L) * dD1) * i1;
    d[4] = 2.0 * tau * (1.0 * D1 - (4.0 + L) * dD1) * i1;
    d[5] = tau * ((3.0 + 2.0 * L) * D1 - (4.0 + L * (3.0 + L)) * dD1) * i1;
}

// acc[s] += dL/dkappa_s, acc[2+s] += dL/dalpha_s from the coefficient cotangents cb[6]
// of species s at mode (kx, ky, kz).
template <typename T>
__device__ __forceinline__ void coef_grad(const ColArgs<T>& a, int s, int kx, int ky, int kz, const double* cb,
                                          double* acc) {
    const double Lam = a.lam[0][kx] + a.lam[1][ky] + a.lam[2][kz];
    if (!(Lam > 0.0)) return;                     // L = 0 for every kappa and alpha
    const double Lf = pow(Lam, 0.5 * a.alpha[s]);
    double d[6];
    if (a.scheme == SFRD_SCHEME_COX_MATTHEWS) cm_dcoef_dL(a.kappa[s] * a.tau * Lf, a.tau, d);
    else dcoef_dL(a.kappa[s] * a.tau * Lf, a.tau, d);
    double G = 0.0;
#pragma unroll
    for (int q = 0; q < 6; ++q) G += cb[q] * d[q];
    acc[s] += G * a.tau * Lf;
    acc[2 + s] += G * a.kappa[s] * a.tau * Lf * 0.5 * log(Lam);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

template <int NV>
__device__ __forceinline__ void flush_sums(const double* acc, double* dst) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        const double v = warp_sum(acc[q]);
        if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst + q, v);
    }
}

}  // namespace v2
}  // namespace sfrd
