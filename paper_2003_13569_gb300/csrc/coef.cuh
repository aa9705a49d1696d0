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

// Cox-Matthews ETDRK4 coefficients (exact exponentials), z = -L <= 0, in the places of the six
// arrays above: R13 -> e^z, Q13 -> e^{z/2}, phi -> (tau/2) psi1(z/2),
// phi1 -> tau (psi1 - 3 psi2 + 4 psi3), phi2 -> 2 tau (psi2 - 2 psi3), phi3 -> tau (-psi2 + 4 psi3),
// with psi_k(z) = sum_{n >= 0} z^n / (n + k)! the phi-functions of exponential integrators.  For
// |z| < 1 the psi_k are summed from their Taylor series (20 terms: the remainder is below 1e-19);
// for |z| >= 1 the closed forms e.g. phi1 = tau [-4 - z + e^z (4 - 3z + z^2)] / z^3 are used, whose
// cancellation is at most a factor ~150 there.  FP64.
constexpr double cm_inv_fact(int m) {
    double r = 1.0;
    for (int i = 2; i <= m; ++i) r /= (double)i;
    return r;
}
#define SFRD_IF4(m) cm_inv_fact(m), cm_inv_fact(m + 1), cm_inv_fact(m + 2), cm_inv_fact(m + 3)
static __constant__ double kCmInvFact[24] = {SFRD_IF4(0), SFRD_IF4(4), SFRD_IF4(8), SFRD_IF4(12), SFRD_IF4(16),
                                             SFRD_IF4(20)};
#undef SFRD_IF4

// sum_{n=0}^{19} z^n / (n+k)!, Horner from the highest term (k <= 3)
__device__ inline double cm_series(double z, int k) {
    double acc = kCmInvFact[19 + k];
    for (int n = 18; n >= 0; --n) acc = acc * z + kCmInvFact[n + k];
    return acc;
}

__device__ inline void cm_coefficients(double L, double tau, double& R, double& Q, double& phi,
                                                double& p1, double& p2, double& p3) {
    const double z = -L, w = -0.5 * L;
    R = exp(z);
    Q = exp(w);
    phi = 0.5 * tau * (w > -1.0 ? cm_series(w, 1) : (Q - 1.0) / w);
    if (z > -1.0) {
        const double s1 = cm_series(z, 1), s2 = cm_series(z, 2), s3 = cm_series(z, 3);
        p1 = tau * (s1 - 3.0 * s2 + 4.0 * s3);
        p2 = 2.0 * tau * (s2 - 2.0 * s3);
        p3 = tau * (-s2 + 4.0 * s3);
    } else {
        const double z3 = z * z * z;
        p1 = tau * (-4.0 - z + R * (4.0 - 3.0 * z + z * z)) / z3;
        p2 = 2.0 * tau * (2.0 + z + R * (z - 2.0)) / z3;
        p3 = tau * (-4.0 - 3.0 * z - z * z + R * (4.0 - z)) / z3;
    }
}

// psi_0..psi_4 at z <= 0: Taylor series for |z| < 1, else psi_0 = e^z and the recurrence
// psi_{k+1} = (psi_k - 1/k!) / z (each step divides by |z| >= 1: absolute errors do not grow).
__device__ inline void cm_psi(double z, double* ps) {
    if (z > -1.0) {
#pragma unroll
        for (int k = 0; k <= 4; ++k) ps[k] = cm_series(z, k);
    } else {
        ps[0] = exp(z);
#pragma unroll
        for (int k = 0; k < 4; ++k) ps[k + 1] = (ps[k] - kCmInvFact[k]) / z;
    }
}

// dC/dL of the Cox-Matthews coefficients, order R, Q, phi, phi1, phi2, phi3 (the slots of
// R13, Q13, phi, phi1, phi2, phi3).  With z = -L (dz/dL = -1) and psi_k' = psi_k - k psi_{k+1}
// (term-by-term from the series):
//   d e^z = e^z;  d[(tau/2) psi1(z/2)]/dz = (tau/4)(psi1 - psi2)(z/2);
//   phi1' = tau (psi1 - 4 psi2 + 10 psi3 - 12 psi4),  phi2' = 2 tau (psi2 - 4 psi3 + 6 psi4),
//   phi3' = tau (-psi2 + 6 psi3 - 12 psi4)   (derivatives in z).
__device__ inline void cm_dcoef_dL(double L, double tau, double* d) {
    double ps[5], pw[5];
    cm_psi(-L, ps);
    cm_psi(-0.5 * L, pw);
    d[0] = -ps[0];
    d[1] = -0.5 * pw[0];
    d[2] = -0.25 * tau * (pw[1] - pw[2]);
    d[3] = -tau * (ps[1] - 4.0 * ps[2] + 10.0 * ps[3] - 12.0 * ps[4]);
    d[4] = -2.0 * tau * (ps[2] - 4.0 * ps[3] + 6.0 * ps[4]);
    d[5] = -tau * (-ps[2] + 6.0 * ps[3] - 12.0 * ps[4]);
}

}  // namespace sfrd
