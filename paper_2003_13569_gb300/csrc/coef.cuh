// Padé(1,3) exponential time differencing coefficients as rational functions of L = kappa tau
// Lambda^{alpha/2} (Algorithm 1, precompute lines; R13 of Eq. 37 and the phi-functions of the
// ETDRK4-P13 stages with e^{-z} replaced by R13).  With
//   D1 = 24 + 18 L + 6 L^2 + L^3   and   D2 = 192 + 72 L + 12 L^2 + L^3  (= 8 times D1 at L/2),
//   R13 = (24 - 6 L) / D1,  phi1 = tau (4 - L) / D1,  phi2 = 2 tau (4 + L) / D1,
//   phi3 = tau (4 + 3 L + L^2) / D1,  Q13 = R13(L/2) = 24 (8 - L) / D2,
//   phi = tau (96 + 12 L + L^2) / D2.
// For L >= 0 every denominator is positive and no term cancels as L -> 0, so the forms keep the
// working precision's relative accuracy (the numerators 24 - 6L, 8 - L, 4 - L change sign away from
// 0, where only the absolute error is small, at the coefficient's own scale).
#pragma once

namespace sfrd {

template <typename T>
__host__ __device__ __forceinline__ void p13_qphi(T L, T tau, T& Q, T& phi) {
    const T D2 = (T)192 + L * ((T)72 + L * ((T)12 + L));
    const T r = (T)1 / D2;
    Q = (T)24 * ((T)8 - L) * r;
    phi = tau * ((T)96 + L * ((T)12 + L)) * r;
}

template <typename T>
__host__ __device__ __forceinline__ void p13_rphi(T L, T tau, T& R, T& p1, T& p2, T& p3) {
    const T D1 = (T)24 + L * ((T)18 + L * ((T)6 + L));
    const T r = (T)1 / D1;
    R = ((T)24 - (T)6 * L) * r;
    p1 = tau * ((T)4 - L) * r;
    p2 = (T)2 * tau * ((T)4 + L) * r;
    p3 = tau * ((T)4 + L * ((T)3 + L)) * r;
}

}  // namespace sfrd
