// Pointwise reaction terms f(u, t) evaluated inside the contiguous-axis pass.
#pragma once

#include "sfrd_internal.h"

namespace sfrd {

// ---- reaction terms (Section 5.2; parameters as documented in sfrd.h) -----------

// `kind` is passed separately so that a caller can give a compile-time constant
// and have the switch folded away.
template <typename T>
__device__ __forceinline__ void react2k(int kind, const ReactDev& re, T u, T v, T& fu, T& fv) {
    switch (kind) {
        case SFRD_REACT_FHN: {
            const T mu = (T)re.p[0], eps = (T)re.p[1], beta = (T)re.p[2], gam = (T)re.p[3], del = (T)re.p[4];
            fu = u * ((T)1 - u) * (u - mu) - v;
            fv = eps * (beta * u - gam * v - del);
        } break;
        case SFRD_REACT_GRAY_SCOTT: {
            const T F = (T)re.p[0], K = (T)re.p[1];
            const T uvv = u * v * v;
            fu = -uvv + F * ((T)1 - u);
            fv = uvv - (F + K) * v;
        } break;
        case SFRD_REACT_SCHNAKENBERG: {
            // f at (U, V) = (u0 + u, v0 + v), the perturbation (u, v) about the offset: with
            // q = U^2 V - u0^2 v0 = v0 u (2 u0 + u) + v U^2,
            //   f_u = g (a - U + U^2 V) = g (c0 - u + q),   f_v = g (b - U^2 V) = g (c1 - q),
            // c0 = a - u0 + u0^2 v0 and c1 = b - u0^2 v0 taken in FP64 at plan time (both zero at the
            // homogeneous steady state).  Every term is of the size of the perturbation, so the
            // O(1) parts of a - U + U^2 V do not cancel in the run precision.
            const T g = (T)re.p[0], u0 = (T)re.off[0], v0 = (T)re.off[1];
            const T U = u0 + u;
            const T q = v0 * u * ((T)2 * u0 + u) + v * U * U;
            fu = g * ((T)re.c[0] - u + q);
            fv = g * ((T)re.c[1] - q);
        } break;
        case SFRD_REACT_GIERER_MEINHARDT: {
            const T U = u + (T)re.off[0], V = v + (T)re.off[1];
            fu = (T)re.p[0] * U * U / V - (T)re.p[1] * U;
            fv = (T)re.p[2] * U * U - (T)re.p[3] * V;
        } break;
        case SFRD_REACT_LINEAR:
            fu = (T)re.p[0] * u;
            fv = (T)re.p[0] * v;
            break;
        default:
            fu = 0;
            fv = 0;
    }
}

template <typename T>
__device__ __forceinline__ void react2(const ReactDev& re, T u, T v, T& fu, T& fv) {
    react2k<T>(re.kind, re, u, v, fu, fv);
}

// Single-species terms; x, y are node coordinates, t the stage time.
template <typename T>
__device__ __forceinline__ T react1(const ReactDev& re, T u, double x, double y, double t) {
    switch (re.kind) {
        case SFRD_REACT_LINEAR:
            return (T)re.p[0] * u;
        case SFRD_REACT_HUXLEY_MMS: {
            // Example 2: exact solution t^alpha cos^3(2 pi x) cos^3(2 pi y); p = [alpha, k1..k4]
            // with Phi = k1 c1x c1y + k2 c3x c1y + k3 c1x c3y + k4 c3x c3y, cNz = cos(2 N pi z).
            const double al = re.p[0];
            const double c1x = cospi(2.0 * x), c1y = cospi(2.0 * y);
            const double c3x = cospi(6.0 * x), c3y = cospi(6.0 * y);
            const double g = c1x * c1x * c1x * c1y * c1y * c1y;
            const double Phi = re.p[1] * c1x * c1y + re.p[2] * c3x * c1y + re.p[3] * c1x * c3y + re.p[4] * c3x * c3y;
            const double ta = t > 0 ? pow(t, al) : 0.0;
            const double dta = t > 0 ? al * pow(t, al - 1.0) : 0.0;
            const double w = ta * g;
            const double src = dta * g + ta * Phi - w * (1.0 - w) * (w - 1.0);
            return u * ((T)1 - u) * (u - (T)1) + (T)src;
        }
        case SFRD_REACT_FISHER_MMS: {
            // Example 1: exact solution e^{-t} sin^3(2 pi x); p = [k1, k3] with the fractional
            // source (kappa/4) e^{-t} (k1 sin 2 pi x - k3 sin 6 pi x), k1 = 3 (2 pi)^alpha, k3 = (6 pi)^alpha
            // folded in (p0 = kappa/4 k1, p1 = kappa/4 k3)
            const double s1 = sinpi(2.0 * x), s3 = sinpi(6.0 * x);
            const double e = exp(-t), sc = s1 * s1 * s1;
            const double src = -2.0 * e * sc + e * (re.p[0] * s1 - re.p[1] * s3) + e * e * sc * sc;
            return u - u * u + (T)src;
        }
        default:
            return 0;
    }
}

// ---- transposed Jacobians and parameter derivatives (for the discrete adjoint) -------
//
// (gu, gv) = J_f(u, v)^T (yu, yv), and dp[q] += w * sum_s (d f_s / d p_q) y_s for the
// parameter vector p of the reaction kind (order as in sfrd.h).
template <typename T>
__device__ __forceinline__ void react2_vjp(const ReactDev& re, T u, T v, T yu, T yv, T& gu, T& gv, double w,
                                           double* dp) {
    switch (re.kind) {
        case SFRD_REACT_FHN: {
            const T mu = (T)re.p[0], eps = (T)re.p[1], beta = (T)re.p[2], gam = (T)re.p[3], del = (T)re.p[4];
            const T fuu = -(T)3 * u * u + (T)2 * ((T)1 + mu) * u - mu;
            gu = fuu * yu + eps * beta * yv;
            gv = -yu - eps * gam * yv;
            dp[0] += w * (double)(-u * ((T)1 - u) * yu);                   // d f_u / d mu
            dp[1] += w * (double)((beta * u - gam * v - del) * yv);        // d f_v / d eps
            dp[2] += w * (double)(eps * u * yv);                            // d f_v / d beta
            dp[3] += w * (double)(-eps * v * yv);                           // d f_v / d gamma
            dp[4] += w * (double)(-eps * yv);                               // d f_v / d delta
        } break;
        case SFRD_REACT_GRAY_SCOTT: {
            const T F = (T)re.p[0], K = (T)re.p[1];
            gu = (-v * v - F) * yu + v * v * yv;
            gv = (-(T)2 * u * v) * yu + ((T)2 * u * v - (F + K)) * yv;
            dp[0] += w * (double)(((T)1 - u) * yu - v * yv);
            dp[1] += w * (double)(-v * yv);
        } break;
        case SFRD_REACT_SCHNAKENBERG: {
            const T g = (T)re.p[0];
            const T U = u + (T)re.off[0], V = v + (T)re.off[1];
            gu = g * (-(T)1 + (T)2 * U * V) * yu - g * (T)2 * U * V * yv;
            gv = g * U * U * yu - g * U * U * yv;
            const T q = (T)re.off[1] * u * ((T)2 * (T)re.off[0] + u) + v * U * U;   // as in react2k
            dp[0] += w * (double)(((T)re.c[0] - u + q) * yu + ((T)re.c[1] - q) * yv);
            dp[1] += w * (double)(g * yu);
            dp[2] += w * (double)(g * yv);
        } break;
        case SFRD_REACT_GIERER_MEINHARDT: {
            const T c1 = (T)re.p[0], c2 = (T)re.p[1], c3 = (T)re.p[2], c4 = (T)re.p[3];
            const T U = u + (T)re.off[0], V = v + (T)re.off[1];
            gu = ((T)2 * c1 * U / V - c2) * yu + (T)2 * c3 * U * yv;
            gv = (-c1 * U * U / (V * V)) * yu - c4 * yv;
            dp[0] += w * (double)(U * U / V * yu);
            dp[1] += w * (double)(-U * yu);
            dp[2] += w * (double)(U * U * yv);
            dp[3] += w * (double)(-V * yv);
        } break;
        case SFRD_REACT_LINEAR:
            gu = (T)re.p[0] * yu;
            gv = (T)re.p[0] * yv;
            dp[0] += w * (double)(u * yu + v * yv);
            break;
        default:
            gu = 0;
            gv = 0;
    }
}

template <typename T>
__device__ __forceinline__ T react1_vjp(const ReactDev& re, T u, T y, double w, double* dp) {
    switch (re.kind) {
        case SFRD_REACT_LINEAR:
            dp[0] += w * (double)(u * y);
            return (T)re.p[0] * y;
        case SFRD_REACT_HUXLEY_MMS:
            return ((T)1 - u) * ((T)3 * u - (T)1) * y;   // d/du [u (1-u)(u-1)]; the source has no u
        case SFRD_REACT_FISHER_MMS:
            return ((T)1 - (T)2 * u) * y;
        default:
            return 0;
    }
}

}  // namespace sfrd
