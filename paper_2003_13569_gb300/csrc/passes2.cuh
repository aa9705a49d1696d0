// Transform passes on the register FFT engine (power-of-two axis lengths).
// Same pass structure, modes and arguments as passes.cuh; the per-axis real
// transform is the length-N packed FFT of fft2.cuh instead of the generic
// shared-memory FFT on the 2N extension.
#pragma once

#include <type_traits>

#include "coef.cuh"
#include "fft2.cuh"
#include "reaction.cuh"

namespace sfrd {
namespace v2 {

// Complex values a thread holds in one FFT step: the larger of step 1 (R1 per owner n2) and step 2
// (R2 per owner k1) over the tile's groups.
template <typename T, int N>
constexpr int fft_values() {
    constexpr int G = kThreads / cc_for(sizeof(T) == 8, N);
    constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
    constexpr int v1 = (R2 + G - 1) / G * R1, v2 = (R1 + G - 1) / G * R2;
    return v1 > v2 ? v1 : v2;
}

// Blocks per SM the register allocation is sized for.  FP32: 64 registers per thread when a thread
// holds at most 16 complex values per FFT step (80 for the update pass, whose batches carry eight
// values per element), 80 up to 20 values, 128 beyond (the 24- and 32-value steps of 384-1024).
// FP64: 128 registers up to 20 values, 255 beyond.
template <typename T, int N, int MODE>
constexpr int min_blocks() {
    return sizeof(T) == 8 ? (fft_values<T, N>() > 20 ? 1 : 2)
                          : (fft_values<T, N>() > 20 ? 2
                                                     : (fft_values<T, N>() > 16 || MODE == MODE_TD ? 3 : 4));
}

template <typename T, int N, int BCT = -1>
struct TileOf {
    static constexpr int CC = TileCC<T, N>::value;
    using E = Eng<T, N, CC, BCT>;
};

// Lengths whose passes are also compiled with the boundary condition fixed at compile time.
template <typename T, int N> struct BcSpecialised { static constexpr bool value = sizeof(T) == 4 && N == 256; };

// Unknowns along an axis of N intervals: N (periodic), N - 1 (Dirichlet), N + 1 (Neumann); taken
// from the runtime axis descriptor when the boundary condition is not fixed at compile time.
template <int N, int BCT>
__device__ __forceinline__ int unknowns(int n_runtime) {
    return BCT == SFRD_BC_PERIODIC ? N : (BCT == SFRD_BC_DIRICHLET ? N - 1 : (BCT == SFRD_BC_NEUMANN ? N + 1 : n_runtime));
}

// RAT: the combination evaluates the coefficients from L (rational-coefficient mode).
// PAIR (FP32 slow-axis stage passes): lines A and B are the adjacent columns x, x + 1 of the species
// bz (ColArgs::cstride == 2, internal arrays), so every element access of the combination is one
// 8-byte pair (16 bytes for the coefficient pairs, 2 x 16 for the quads; 8 bytes of L with RAT).
template <typename T, int N, int MODE, int BCT = -1, bool RAT = false, bool PAIR = false>
__device__ __forceinline__ void col2_body(const ColArgs<T>& a, int bx, int by, unsigned char* smem_raw, int bz = 0) {
    constexpr int CC = TileOf<T, N>::CC;
    using E = typename TileOf<T, N, BCT>::E;
    using C = typename E::C;
    constexpr int LD = E::LD, G = E::G;
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* red = buf + E::ROWS * LD;
    C* red2 = red + G * CC;
    C* tws = red2 + G * CC;
    if (MODE == MODE_PLAIN || MODE == MODE_TD) __builtin_assume(threadIdx.x < kThreads);
    const int tid = threadIdx.x, c = tid % CC, g = tid / CC;
    const AxisDev& ax = a.ax;
    const int n = unknowns<N, BCT>(ax.n), bc = ax.bc;
    const C* tw = static_cast<const C*>(ax.tw);
    const int twstride = bc == SFRD_BC_PERIODIC ? 1 : 2;
    for (int i = tid; i < N * twstride; i += kThreads) tws[i] = __ldg(tw + i);   // visible after the first barrier
    const int xA = bx * a.xw + c * a.cstride, xB = xA + a.bshift;
    // Element indices: one 64-bit tile origin per thread, then 32-bit offsets (every array of the
    // pass holds fewer than 2^32 elements; checked when the plan is made).
    const size_t org_in = (size_t)by * (size_t)a.in_sOther + (size_t)xA + (size_t)bz * (size_t)a.in_sp;
    const size_t org_out = (size_t)by * (size_t)a.out_sOther + (size_t)xA + (size_t)bz * (size_t)a.out_sp;
    const unsigned s_in = (unsigned)a.in_sAxis, s_out = (unsigned)a.out_sAxis;
    bool zin = false;   // the buffer holds the pre-processed line (forward_z)

    if constexpr (PAIR) {
        // element pairs (internal arrays, even pitch: x < pitch implies x + 1 < pitch; 8-byte aligned);
        // the lanes of the last tile beyond the pitch hold zeros and store nothing
        constexpr int NL = (E::ROWS + G - 1) / G;
        const bool okx = xA < a.in_xlim;
        const T* pA = a.in + org_in;
        C z[NL];
#pragma unroll
        for (int t = 0; t < NL; ++t) {
            const int i = g + t * G;
            z[t] = czero<C>();
            if (okx && i < n) z[t] = *reinterpret_cast<const C*>(pA + (unsigned)i * s_in);
        }
#pragma unroll
        for (int t = 0; t < NL; ++t) {
            const int i = g + t * G;
            if (i < n) buf[i * LD + c] = z[t];
        }
    } else if (MODE == MODE_PLAIN && a.bshift == CC && a.in_offB == (long long)CC) {
        // lines A and B are the columns x and x + CC of one array: a tile row is 2 CC consecutive
        // values, read by one warp instruction (LW lanes per row) and stored to the .x (A) or .y (B)
        // halves of the row; all loads of this thread are issued before any shared-memory store
        constexpr int LW = 2 * CC, RPI = 32 / LW, NW = kThreads / 32;
        constexpr int NRW = (E::ROWS + NW * RPI - 1) / (NW * RPI);
        const int w = tid >> 5, l = tid & 31, col = l % LW, sub = l / LW;
        const int x = bx * a.xw + col;
        const bool okx = x < a.in_xlim;
        const T* p = a.in + ((size_t)by * (size_t)a.in_sOther + (size_t)x);
        T* const dst = reinterpret_cast<T*>(buf) + 2 * (col % CC) + col / CC;
        T v[NRW];
#pragma unroll
        for (int r = 0; r < NRW; ++r) {
            const int i = (w * RPI + sub) + r * NW * RPI;
            v[r] = (okx && i < n) ? p[(unsigned)i * s_in] : (T)0;
        }
#pragma unroll
        for (int r = 0; r < NRW; ++r) {
            const int i = (w * RPI + sub) + r * NW * RPI;
            if (i < n) dst[2 * i * LD] = v[r];
        }
    } else if (MODE == MODE_PLAIN && a.cstride == 2) {
        // lines A and B are the adjacent columns x, x + 1: one 2-element load per row where aligned.
        // Each thread loads the mirror pairs (j, N - j), j = g, g + G, ..., N/2, and writes their
        // pre-processed values z_j, z_{N-j}, so the transform reads every value once.
        constexpr int NP = (N / 2 + 1 + G - 1) / G;
        const bool okA = xA < a.in_xlim, okB = xB < a.in_xlim;
        const T* pA = a.in + org_in;
        const bool vec = okB && ((a.in_sAxis | a.in_sOther) & 1) == 0 &&
                         (reinterpret_cast<uintptr_t>(a.in) % sizeof(C)) == 0;
        const int bcx = E::bcv(bc);
        // value at transform index q (0 <= q <= N): unknown q - 1 (Dirichlet, zero at q = 0, N), else q
        auto val = [&](int q) {
            const int i = bcx == SFRD_BC_DIRICHLET ? q - 1 : q;
            C z = czero<C>();
            if (i >= 0 && i < n) {
                const unsigned o = (unsigned)i * s_in;
                if (vec) {
                    z = *reinterpret_cast<const C*>(pA + o);
                } else {
                    z.x = okA ? pA[o] : (T)0;
                    z.y = okB ? pA[o + 1] : (T)0;
                }
            }
            return z;
        };
        C xj[NP], xm[NP];
#pragma unroll
        for (int t = 0; t < NP; ++t) {
            const int j = g + t * G;
            xj[t] = czero<C>();
            xm[t] = czero<C>();
            if (j <= N / 2) {
                xj[t] = val(j);
                xm[t] = val(N - j);
            }
        }
        C anchor = czero<C>();
        // (cos, -sin)(j pi / N) for j = g + t G: the table value at g rotated through the compile-time
        // angle t G pi / N (one table read per thread)
        const C wg = bcx == SFRD_BC_PERIODIC ? czero<C>() : __ldg(tw + g);
        static_for<0, NP>([&](auto TT) {
            constexpr int t = decltype(TT)::value;
            const int j = g + t * G;
            if (j <= N / 2) {
                constexpr T cr = (T)ce_cs2pi(t * G, 2 * N).c, ci = (T)(-ce_cs2pi(t * G, 2 * N).s);
                C w;
                w.x = wg.x * cr - wg.y * ci;
                w.y = wg.x * ci + wg.y * cr;
                C zj, zm;
                E::pre_pair(bc, j, xj[t], xm[t], -w.y, w.x, zj, zm, anchor);
                buf[j * LD + c] = zj;
                if (j > 0 && j < N / 2) buf[(N - j) * LD + c] = zm;
            }
        });
        red2[g * CC + c] = anchor;
        zin = true;
    } else if (MODE == MODE_PLAIN && a.cstride == 2) {
        // lines A and B are the adjacent columns x, x + 1: one 2-element load per row where aligned
        constexpr int NL = (E::ROWS + G - 1) / G;
        const bool okA = xA < a.in_xlim, okB = xB < a.in_xlim;
        const T* pA = a.in + org_in;
        const bool vec = okB && ((a.in_sAxis | a.in_sOther) & 1) == 0 &&
                         (reinterpret_cast<uintptr_t>(a.in) % sizeof(C)) == 0;
        C z[NL];
#pragma unroll
        for (int t = 0; t < NL; ++t) {
            const int i = g + t * G;
            const unsigned o = (unsigned)i * s_in;
            if (i < n && vec) {
                z[t] = *reinterpret_cast<const C*>(pA + o);
            } else {
                z[t].x = (okA && i < n) ? pA[o] : (T)0;
                z[t].y = (okB && i < n) ? pA[o + 1] : (T)0;
            }
        }
#pragma unroll
        for (int t = 0; t < NL; ++t) {
            const int i = g + t * G;
            if (i < n) buf[i * LD + c] = z[t];
        }
    } else {
        // all loads of this thread issued before any shared-memory store
        constexpr int NL = (E::ROWS + G - 1) / G;
        const bool okA = xA < a.in_xlim, okB = xB < a.in_xlim;
        const T* pA = a.in + org_in;
        const unsigned oB = (unsigned)a.in_offB;
        C z[NL];
#pragma unroll
        for (int t = 0; t < NL; ++t) {
            const int i = g + t * G;
            const unsigned o = (unsigned)i * s_in;
            z[t].x = (okA && i < n) ? pA[o] : (T)0;
            z[t].y = (okB && i < n) ? pA[o + oB] : (T)0;
        }
#pragma unroll
        for (int t = 0; t < NL; ++t) {
            const int i = g + t * G;
            if (i < n) buf[i * LD + c] = z[t];
        }
    }
    __syncthreads();
    if (zin) E::forward_z(buf, bc, tws, twstride, c, g);
    else E::forward(buf, red2, bc, tws, twstride, c, g);

    if (MODE == MODE_PLAIN && a.cstride == 2) {
        // adjacent columns: one 2-element store per output where aligned
        const bool okA = xA < a.out_xlim, okB = xB < a.out_xlim;
        T* qA = a.out + org_out;
        const bool vec = okB && ((a.out_sAxis | a.out_sOther) & 1) == 0 &&
                         (reinterpret_cast<uintptr_t>(a.out) % sizeof(C)) == 0;
        const T sc = (T)a.scale;
        E::post(buf, red, red2, bc, c, g, [&](int i, C v) {
            const unsigned o = (unsigned)i * s_out;
            if (vec) {
                C w;
                w.x = v.x * sc;
                w.y = v.y * sc;
                *reinterpret_cast<C*>(qA + o) = w;
            } else {
                if (okA) qA[o] = v.x * sc;
                if (okB) qA[o + 1] = v.y * sc;
            }
        });
        return;
    }
    if (MODE == MODE_PLAIN) {
        const bool okA = xA < a.out_xlim, okB = xB < a.out_xlim;
        T* qA = a.out + org_out;
        const unsigned oB = (unsigned)a.out_offB;
        const T sc = (T)a.scale;
        E::post(buf, red, red2, bc, c, g, [&](int i, C v) {
            const unsigned o = (unsigned)i * s_out;
            if (okA) qA[o] = v.x * sc;
            if (okB) qA[o + oB] = v.y * sc;
        });
        return;
    }

    {
        const bool okA = xA < a.in_xlim, okB = xB < a.in_xlim;
        const unsigned e0 = (unsigned)org_in, eoB = (unsigned)a.in_offB;
        const T invC = (T)a.invC;
        // values read by the combination: batch-loaded (all loads of a batch before any use)
        using V2 = typename Cx<T>::type;                                    // (Q13, phi) pair
        constexpr int NV = MODE == MODE_TD ? 8 : (MODE == MODE_TC ? 4 : (MODE == MODE_T0 ? 1 : 3));
        constexpr int B = 1;
        T ld[2 * B][2][NV];
        const bool ok[2] = {okA, okB};
        const unsigned clB = (unsigned)a.clB;
        const unsigned clsub = PAIR && RAT ? (unsigned)((long long)bz * (a.in_sp - a.cl_sp)) : 0u;
        auto pre = [&](int slot, int k) {
            const unsigned eA = e0 + (unsigned)k * s_in;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ok[h]) continue;
                const unsigned i = eA + (h ? eoB : 0u);
                // read-only inputs through the non-coherent path (every element is read once,
                // before its own update); coefficient pairs and quads as single vector loads
                if constexpr (PAIR) {
                    if (h || !ok[0]) continue;   // both lines at once
                    if constexpr (RAT) {
                        const float2 l = __ldg(reinterpret_cast<const float2*>(a.CL + (eA - clsub)));
                        const float2 u = __ldg(reinterpret_cast<const float2*>(a.U + eA));
                        if (MODE == MODE_TD) {
                            const float2 f1 = __ldg(reinterpret_cast<const float2*>(a.F1 + eA));
                            const float2 f2 = __ldg(reinterpret_cast<const float2*>(a.F2 + eA));
                            const float2 f3 = __ldg(reinterpret_cast<const float2*>(a.F3 + eA));
                            ld[slot][0][4] = l.x; ld[slot][1][4] = l.y;
                            ld[slot][0][0] = u.x; ld[slot][1][0] = u.y;
                            ld[slot][0][1] = f1.x; ld[slot][1][1] = f1.y;
                            ld[slot][0][2] = f2.x; ld[slot][1][2] = f2.y;
                            ld[slot][0][3] = f3.x; ld[slot][1][3] = f3.y;
                        } else if (MODE != MODE_T0) {
                            ld[slot][0][0] = l.x; ld[slot][1][0] = l.y;
                            ld[slot][0][2] = u.x; ld[slot][1][2] = u.y;
                            if (MODE == MODE_TC) {
                                const float2 f1 = __ldg(reinterpret_cast<const float2*>(a.F1 + eA));
                                ld[slot][0][3] = f1.x; ld[slot][1][3] = f1.y;
                            }
                        }
                    } else if (MODE == MODE_TA || MODE == MODE_TB || MODE == MODE_TC) {
                        const float4 q = __ldg(reinterpret_cast<const float4*>(a.CQ + 2 * (size_t)eA));
                        const float2 u = __ldg(reinterpret_cast<const float2*>(a.U + eA));
                        ld[slot][0][0] = q.x; ld[slot][0][1] = q.y; ld[slot][1][0] = q.z; ld[slot][1][1] = q.w;
                        ld[slot][0][2] = u.x; ld[slot][1][2] = u.y;
                        if (MODE == MODE_TC) {
                            const float2 f1 = __ldg(reinterpret_cast<const float2*>(a.F1 + eA));
                            ld[slot][0][3] = f1.x; ld[slot][1][3] = f1.y;
                        }
                    } else if (MODE == MODE_TD) {
                        const float4 r0 = __ldg(reinterpret_cast<const float4*>(a.CR + 4 * (size_t)eA));
                        const float4 r1 = __ldg(reinterpret_cast<const float4*>(a.CR + 4 * (size_t)eA) + 1);
                        const float2 u = __ldg(reinterpret_cast<const float2*>(a.U + eA));
                        const float2 f1 = __ldg(reinterpret_cast<const float2*>(a.F1 + eA));
                        const float2 f2 = __ldg(reinterpret_cast<const float2*>(a.F2 + eA));
                        const float2 f3 = __ldg(reinterpret_cast<const float2*>(a.F3 + eA));
                        ld[slot][0][4] = r0.x; ld[slot][0][5] = r0.y; ld[slot][0][6] = r0.z; ld[slot][0][7] = r0.w;
                        ld[slot][1][4] = r1.x; ld[slot][1][5] = r1.y; ld[slot][1][6] = r1.z; ld[slot][1][7] = r1.w;
                        ld[slot][0][0] = u.x; ld[slot][1][0] = u.y;
                        ld[slot][0][1] = f1.x; ld[slot][1][1] = f1.y;
                        ld[slot][0][2] = f2.x; ld[slot][1][2] = f2.y;
                        ld[slot][0][3] = f3.x; ld[slot][1][3] = f3.y;
                    }
                } else if (RAT) {
                    const T Lraw = __ldg(a.CL + eA + (h ? clB : 0u));
                    if (MODE == MODE_TD) {
                        ld[slot][h][4] = Lraw;
                        ld[slot][h][0] = __ldg(a.U + i);
                        ld[slot][h][1] = __ldg(a.F1 + i);
                        ld[slot][h][2] = __ldg(a.F2 + i);
                        ld[slot][h][3] = __ldg(a.F3 + i);
                    } else if (MODE != MODE_T0) {
                        ld[slot][h][0] = Lraw;
                        ld[slot][h][2] = __ldg(a.U + i);
                        if (MODE == MODE_TC) ld[slot][h][3] = __ldg(a.F1 + i);
                    }
                } else if (MODE == MODE_TA || MODE == MODE_TB || MODE == MODE_TC) {
                    const V2 q = __ldg(reinterpret_cast<const V2*>(a.CQ) + i);
                    ld[slot][h][0] = q.x;
                    ld[slot][h][1] = q.y;
                    ld[slot][h][2] = __ldg(a.U + i);
                    if (MODE == MODE_TC) ld[slot][h][3] = __ldg(a.F1 + i);
                } else if (MODE == MODE_TD) {
                    if (sizeof(T) == 4) {
                        const float4 r = __ldg(reinterpret_cast<const float4*>(a.CR) + i);
                        ld[slot][h][4] = (T)r.x;
                        ld[slot][h][5] = (T)r.y;
                        ld[slot][h][6] = (T)r.z;
                        ld[slot][h][7] = (T)r.w;
                    } else {
                        const double2* cr = reinterpret_cast<const double2*>(a.CR) + 2 * (size_t)i;
                        const double2 r0 = __ldg(cr);
                        const double2 r1 = __ldg(cr + 1);
                        ld[slot][h][4] = (T)r0.x;
                        ld[slot][h][5] = (T)r0.y;
                        ld[slot][h][6] = (T)r1.x;
                        ld[slot][h][7] = (T)r1.y;
                    }
                    ld[slot][h][0] = __ldg(a.U + i);
                    ld[slot][h][1] = __ldg(a.F1 + i);
                    ld[slot][h][2] = __ldg(a.F2 + i);
                    ld[slot][h][3] = __ldg(a.F3 + i);
                }
            }
        };
        T* const F4 = a.F4;
        const T lm[2] = {(T)a.cl_mult[0], (T)a.cl_mult[1]};
        const T lmz = (T)a.cl_mult[bz & 1];   // element-pair grid: both lines are species bz
        const T tau = (T)a.tau;
        E::post_b<B>(buf, red, red2, bc, c, g, pre, [&](int slot, int k, C Fv) {
            const unsigned eA = e0 + (unsigned)k * s_in;
            const T F[2] = {Fv.x, Fv.y};
            T s[2] = {0, 0};
            if constexpr (PAIR) {
                T sv[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    T Lc[NV];
#pragma unroll
                    for (int m = 0; m < NV; ++m) Lc[m] = ld[slot][h][m];
                    if (RAT) {
                        if (MODE == MODE_TD) p13_rphi<T>(lmz * Lc[4], tau, Lc[4], Lc[5], Lc[6], Lc[7]);
                        else if (MODE != MODE_T0) p13_qphi<T>(lmz * Lc[0], tau, Lc[0], Lc[1]);
                    }
                    const T* L = Lc;
                    if (MODE == MODE_TA || MODE == MODE_TB) {
                        sv[h] = L[0] * L[2] + L[1] * F[h];
                    } else if (MODE == MODE_TC) {
                        const T ah = L[0] * L[2] + L[1] * L[3];
                        sv[h] = L[0] * ah + L[1] * ((T)2 * F[h] - L[3]);
                    } else {
                        sv[h] = L[4] * L[0] + L[5] * L[1] + L[6] * (L[2] + L[3]) + L[7] * F[h];
                    }
                }
                const float2 fp = make_float2((float)F[0], (float)F[1]);
                if (!ok[0]) sv[0] = sv[1] = 0;
                if (ok[0] && MODE == MODE_TA) *reinterpret_cast<float2*>(a.F1 + eA) = fp;
                if (ok[0] && MODE == MODE_TB) *reinterpret_cast<float2*>(a.F2 + eA) = fp;
                if (ok[0] && MODE == MODE_TC) *reinterpret_cast<float2*>(a.F3 + eA) = fp;
                if (ok[0] && MODE == MODE_TD) {
                    if (F4) *reinterpret_cast<float2*>(F4 + eA) = fp;
                    *reinterpret_cast<float2*>(a.U + eA) = make_float2((float)sv[0], (float)sv[1]);
                }
                C z;
                z.x = sv[0] * invC;
                z.y = sv[1] * invC;
                buf[k * LD + c] = z;
                return;
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                if (!ok[h]) continue;
                const unsigned i = eA + (h ? eoB : 0u);
                T Lc[NV];
#pragma unroll
                for (int m = 0; m < NV; ++m) Lc[m] = ld[slot][h][m];
                if (RAT) {   // coefficients in place of the stored ones: (Q, phi) or (R, phi1, phi2, phi3)
                    if (MODE == MODE_TD) p13_rphi<T>(lm[h] * Lc[4], tau, Lc[4], Lc[5], Lc[6], Lc[7]);
                    else if (MODE != MODE_T0) p13_qphi<T>(lm[h] * Lc[0], tau, Lc[0], Lc[1]);
                }
                const T* L = Lc;
                if (MODE == MODE_T0) {
                    a.U[i] = F[h];
                    s[h] = F[h];
                } else if (MODE == MODE_TA || MODE == MODE_TB) {
                    if (MODE == MODE_TA) a.F1[i] = F[h]; else a.F2[i] = F[h];
                    s[h] = L[0] * L[2] + L[1] * F[h];
                } else if (MODE == MODE_TC) {
                    a.F3[i] = F[h];
                    const T ah = L[0] * L[2] + L[1] * L[3];
                    s[h] = L[0] * ah + L[1] * ((T)2 * F[h] - L[3]);
                } else {  // MODE_TD: U <- R U + phi1 F1 + phi2 (F2 + F3) + phi3 F4
                    const T un = L[4] * L[0] + L[5] * L[1] + L[6] * (L[2] + L[3]) + L[7] * F[h];
                    if (F4) F4[i] = F[h];
                    a.U[i] = un;
                    s[h] = un;
                }
            }
            C z;
            z.x = s[0] * invC;
            z.y = s[1] * invC;
            buf[k * LD + c] = z;
        });
    }
    __syncthreads();
    E::forward(buf, red2, bc, tws, twstride, c, g);
    if constexpr (PAIR) {
        T* qA = a.out + org_out;
        const bool okx = xA < a.out_xlim;
        E::post(buf, red, red2, bc, c, g, [&](int i, C v) {
            if (okx) *reinterpret_cast<C*>(qA + (unsigned)i * s_out) = v;
        });
    } else {
        const bool okA = xA < a.out_xlim, okB = xB < a.out_xlim;
        T* qA = a.out + org_out;
        const unsigned oB = (unsigned)a.out_offB;
        E::post(buf, red, red2, bc, c, g, [&](int i, C v) {
            const unsigned o = (unsigned)i * s_out;
            if (okA) qA[o] = v.x;
            if (okB) qA[o + oB] = v.y;
        });
    }
    if (MODE == MODE_TD && bx == 0 && by == 0 && bz == 0 && threadIdx.x == 0) a.clock->k += 1;
}

template <typename T, int N, int MODE, int BCT = -1, bool RAT = false, bool PAIR = false>
__global__ void __launch_bounds__(kThreads, (min_blocks<T, N, MODE>())) col2_kernel(const ColArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // The middle-axis pass takes its planes in reverse order: it then starts on those its producer (the
    // slow-axis or the x pass) wrote last, still in L2, and leaves to the next pass the planes that pass
    // reads first (255^3 step -2.7 %: y -5 %, x -2 %, slow-axis stages -2 %).
    const int by = MODE == MODE_PLAIN ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
    col2_body<T, N, MODE, BCT, RAT, PAIR>(a, blockIdx.x, by, smem_raw, blockIdx.z);
}

// The FP32 contiguous-axis pass is also compiled once per two-species reaction kind (KIND >= 0: the
// reaction of that kind only, no stage save), so that the kernel holds one reaction unpacking instead of
// all of them: at length 1024 the unrolled unpackings of every kind exceed the instruction cache, and at
// 256 the kernel of every kind spills under its 64-register budget where the per-kind kernels do not.
template <typename T, int N> struct KindSpecialised { static constexpr bool value = sizeof(T) == 4; };

template <typename T, int N, int MODE, int BCT = -1, int KIND = -1>
__device__ __forceinline__ void x2_body(const XArgs<T>& a, int bx, unsigned char* smem_raw) {
    constexpr int CC = TileOf<T, N>::CC;
    using E = typename TileOf<T, N, BCT>::E;
    using C = typename E::C;
    constexpr int LD = E::LD, G = E::G;
    C* buf = reinterpret_cast<C*>(smem_raw);
    C* red = buf + E::ROWS * LD;
    C* red2 = red + G * CC;
    C* tws = red2 + G * CC;
    __builtin_assume(threadIdx.x < kThreads);
    const int tid = threadIdx.x, c = tid % CC, g = tid / CC;
    const AxisDev& ax = a.ax;
    const int n = unknowns<N, BCT>(ax.n), bc = ax.bc;
    const C* tw = static_cast<const C*>(ax.tw);
    const int twstride = bc == SFRD_BC_PERIODIC ? 1 : 2;
    for (int i = tid; i < N * twstride; i += kThreads) tws[i] = __ldg(tw + i);   // visible after the first barrier
    const int shiftB = (a.S == 2) ? 0 : CC;
    const int r0 = bx * (a.S == 2 ? CC : 2 * CC);

    // transposed load: warp w reads rows w, w + 8, ... ; lane l reads x = l, l + 32, ...
    {
        constexpr int NW = kThreads / 32;               // warps
        constexpr int RW = (CC + NW - 1) / NW;          // rows per warp
        constexpr int XL = (E::ROWS + 31) / 32;         // x per lane
        const int w = tid >> 5, l = tid & 31;
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) {
            const int cc = w + rr * NW;
            const int rA = r0 + cc, rB = rA + shiftB;
            const bool okA = cc < CC && rA < a.rows, okB = cc < CC && rB < a.rows;
            const T* pA = a.in + (long long)rA * a.in_pitch;
            C z[XL];
#pragma unroll
            for (int t = 0; t < XL; ++t) {
                const int x = l + 32 * t;
                z[t].x = (okA && x < n) ? pA[x] : (T)0;
                z[t].y = (okB && x < n) ? pA[a.in_offB + x] : (T)0;
            }
            if (cc < CC) {
#pragma unroll
                for (int t = 0; t < XL; ++t) {
                    const int x = l + 32 * t;
                    if (x < n) buf[x * LD + cc] = z[t];
                }
            }
        }
    }
    __syncthreads();
    E::forward(buf, red2, bc, tws, twstride, c, g);
    if (MODE == MODE_REACT) {
        const int rA = r0 + c, rB = rA + shiftB;
        T* sv = a.save ? a.save + (long long)rA * a.out_pitch : nullptr;   // stage save (adjoint recomputation)
        if constexpr (KIND >= 0) {
            // the launch has checked: two species, no stage save, reaction kind KIND
            E::post(buf, red, red2, bc, c, g, [&](int i, C v) {
                C f;
                react2k<T>(KIND, a.re, v.x, v.y, f.x, f.y);
                buf[i * LD + c] = f;
            });
        } else if (a.S == 2 && !sv) {
            // two-species kinds: the pointwise reaction is applied to each physical value as the
            // transform unpacks it (one unpacking per kind, so that the kind is a compile-time constant)
            auto run = [&](auto kind) {
                E::post(buf, red, red2, bc, c, g, [&](int i, C v) {
                    C f;
                    react2k<T>(decltype(kind)::value, a.re, v.x, v.y, f.x, f.y);
                    buf[i * LD + c] = f;
                });
            };
            switch (a.re.kind) {
                case SFRD_REACT_SCHNAKENBERG: run(std::integral_constant<int, SFRD_REACT_SCHNAKENBERG>()); break;
                case SFRD_REACT_GRAY_SCOTT: run(std::integral_constant<int, SFRD_REACT_GRAY_SCOTT>()); break;
                case SFRD_REACT_FHN: run(std::integral_constant<int, SFRD_REACT_FHN>()); break;
                case SFRD_REACT_GIERER_MEINHARDT: run(std::integral_constant<int, SFRD_REACT_GIERER_MEINHARDT>()); break;
                case SFRD_REACT_LINEAR: run(std::integral_constant<int, SFRD_REACT_LINEAR>()); break;
                default: run(std::integral_constant<int, SFRD_REACT_NONE>()); break;
            }
        } else {
            E::post(buf, red, red2, bc, c, g, [&](int i, C v) { buf[i * LD + c] = v; });
            __syncthreads();
            // pointwise reaction on the physical values, saved for the adjoint recomputation when asked
            const double t = a.clock->t0 + ((double)a.clock->k + a.stage_frac) * a.tau;
#pragma unroll 1
            for (int i = g; i < n; i += G) {
                const C v = buf[i * LD + c];
                if (sv) {
                    if (rA < a.rows) sv[i] = v.x;
                    if (rB < a.rows) sv[a.out_offB + i] = v.y;
                }
                C f;
                if (a.S == 2) {
                    react2<T>(a.re, v.x, v.y, f.x, f.y);
                } else {
                    const double x = ax.lo + (ax.node0 + i) * ax.h;
                    const int yA = rA % a.ny, yB = rB % a.ny;
                    const double ya = a.ay.lo + (a.ay.node0 + yA) * a.ay.h;
                    const double yb = a.ay.lo + (a.ay.node0 + yB) * a.ay.h;
                    f.x = react1<T>(a.re, v.x, x, ya, t);
                    f.y = react1<T>(a.re, v.y, x, yb, t);
                }
                buf[i * LD + c] = f;
            }
        }
        __syncthreads();
        E::forward(buf, red2, bc, tws, twstride, c, g);
    }
    E::post(buf, red, red2, bc, c, g, [&](int i, C v) { buf[i * LD + c] = v; });
    __syncthreads();
    {
        constexpr int NW = kThreads / 32;
        constexpr int RW = (CC + NW - 1) / NW;
        const int w = tid >> 5, l = tid & 31;
        const int xend = a.out_fill > n ? a.out_fill : n;
#pragma unroll
        for (int rr = 0; rr < RW; ++rr) {
            const int cc = w + rr * NW;
            if (cc >= CC) continue;
            const int rA = r0 + cc, rB = rA + shiftB;
            T* qA = a.out + (long long)rA * a.out_pitch;
            for (int x = l; x < xend; x += 32) {
                const C v = x < n ? buf[x * LD + cc] : czero<C>();
                if (rA < a.rows) qA[x] = v.x;
                if (rB < a.rows) qA[a.out_offB + x] = v.y;
            }
        }
    }
}

template <typename T, int N, int MODE, int BCT = -1, int KIND = -1>
__global__ void __launch_bounds__(kThreads, (min_blocks<T, N, MODE>())) x2_kernel(const XArgs<T> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    x2_body<T, N, MODE, BCT, KIND>(a, blockIdx.x, smem_raw);
}

// ---- launch --------------------------------------------------------------------------
//
// The kernels of a length fall into four families, each with its own launch and set-up function, so
// that a translation unit can instantiate one family: the long FP32 lengths compile as several objects
// in parallel.  PLAIN: the column passes of every mode on the default layouts; PAIR (FP32): the stage
// passes on element pairs, stored and rational coefficients; RAT (FP32): the rational-coefficient stage
// passes on the default layouts; X: the contiguous-axis pass.

template <typename T>
cudaError_t set_smem_attrs(void (*k)(const T), int bytes) {
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    return e;
}

constexpr bool is_stage_mode(int mode) {
    return mode == MODE_TA || mode == MODE_TB || mode == MODE_TC || mode == MODE_TD;
}

template <typename T, int N, int BCT>
cudaError_t col2_plain_launch_bc(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    void (*k)(const ColArgs<T>) = nullptr;
    switch (mode) {
        case MODE_PLAIN: k = col2_kernel<T, N, MODE_PLAIN, BCT>; break;
        case MODE_T0: k = col2_kernel<T, N, MODE_T0, BCT>; break;
        case MODE_TA: k = col2_kernel<T, N, MODE_TA, BCT>; break;
        case MODE_TB: k = col2_kernel<T, N, MODE_TB, BCT>; break;
        case MODE_TC: k = col2_kernel<T, N, MODE_TC, BCT>; break;
        default: k = col2_kernel<T, N, MODE_TD, BCT>; break;
    }
    k<<<grid, kThreads, TileOf<T, N>::E::smem_bytes(), s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N, int BCT>
cudaError_t col2_plain_prepare_bc() {
    void (*ks[])(const ColArgs<T>) = {col2_kernel<T, N, MODE_PLAIN, BCT>, col2_kernel<T, N, MODE_T0, BCT>,
                                      col2_kernel<T, N, MODE_TA, BCT>,    col2_kernel<T, N, MODE_TB, BCT>,
                                      col2_kernel<T, N, MODE_TC, BCT>,    col2_kernel<T, N, MODE_TD, BCT>};
    for (auto k : ks) {
        const cudaError_t e = set_smem_attrs(k, kMaxDynSmem2);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Stage passes on element pairs (FP32 only); a.CL selects the rational-coefficient form.
template <typename T, int N, int BCT>
cudaError_t col2_pair_launch_bc(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        void (*k)(const ColArgs<T>) = nullptr;
        if (a.CL) {
            switch (mode) {
                case MODE_TA: k = col2_kernel<T, N, MODE_TA, BCT, true, true>; break;
                case MODE_TB: k = col2_kernel<T, N, MODE_TB, BCT, true, true>; break;
                case MODE_TC: k = col2_kernel<T, N, MODE_TC, BCT, true, true>; break;
                default: k = col2_kernel<T, N, MODE_TD, BCT, true, true>; break;
            }
        } else {
            switch (mode) {
                case MODE_TA: k = col2_kernel<T, N, MODE_TA, BCT, false, true>; break;
                case MODE_TB: k = col2_kernel<T, N, MODE_TB, BCT, false, true>; break;
                case MODE_TC: k = col2_kernel<T, N, MODE_TC, BCT, false, true>; break;
                default: k = col2_kernel<T, N, MODE_TD, BCT, false, true>; break;
            }
        }
        k<<<grid, kThreads, TileOf<T, N>::E::smem_bytes(), s>>>(a);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename T, int N, int BCT>
cudaError_t col2_pair_prepare_bc() {
    if constexpr (sizeof(T) == 4) {
        void (*ks[])(const ColArgs<T>) = {col2_kernel<T, N, MODE_TA, BCT, false, true>,
                                          col2_kernel<T, N, MODE_TB, BCT, false, true>,
                                          col2_kernel<T, N, MODE_TC, BCT, false, true>,
                                          col2_kernel<T, N, MODE_TD, BCT, false, true>,
                                          col2_kernel<T, N, MODE_TA, BCT, true, true>,
                                          col2_kernel<T, N, MODE_TB, BCT, true, true>,
                                          col2_kernel<T, N, MODE_TC, BCT, true, true>,
                                          col2_kernel<T, N, MODE_TD, BCT, true, true>};
        for (auto k : ks) {
            const cudaError_t e = set_smem_attrs(k, kMaxDynSmem2);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Rational-coefficient stage passes on the default layouts (FP32 only).
template <typename T, int N, int BCT>
cudaError_t col2_rat_launch_bc(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        void (*k)(const ColArgs<T>) = nullptr;
        switch (mode) {
            case MODE_TA: k = col2_kernel<T, N, MODE_TA, BCT, true>; break;
            case MODE_TB: k = col2_kernel<T, N, MODE_TB, BCT, true>; break;
            case MODE_TC: k = col2_kernel<T, N, MODE_TC, BCT, true>; break;
            default: k = col2_kernel<T, N, MODE_TD, BCT, true>; break;
        }
        k<<<grid, kThreads, TileOf<T, N>::E::smem_bytes(), s>>>(a);
        return cudaGetLastError();
    } else {
        return cudaErrorInvalidValue;
    }
}

template <typename T, int N, int BCT>
cudaError_t col2_rat_prepare_bc() {
    if constexpr (sizeof(T) == 4) {
        void (*ks[])(const ColArgs<T>) = {col2_kernel<T, N, MODE_TA, BCT, true>, col2_kernel<T, N, MODE_TB, BCT, true>,
                                          col2_kernel<T, N, MODE_TC, BCT, true>, col2_kernel<T, N, MODE_TD, BCT, true>};
        for (auto k : ks) {
            const cudaError_t e = set_smem_attrs(k, kMaxDynSmem2);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// The reaction pass of one two-species kind (the kinds of react2k; any other kind has no reaction there).
template <typename T, int N, int BCT>
void (*x2_kind_kernel(int kind))(const XArgs<T>) {
    switch (kind) {
        case SFRD_REACT_SCHNAKENBERG: return x2_kernel<T, N, MODE_REACT, BCT, SFRD_REACT_SCHNAKENBERG>;
        case SFRD_REACT_GRAY_SCOTT: return x2_kernel<T, N, MODE_REACT, BCT, SFRD_REACT_GRAY_SCOTT>;
        case SFRD_REACT_FHN: return x2_kernel<T, N, MODE_REACT, BCT, SFRD_REACT_FHN>;
        case SFRD_REACT_GIERER_MEINHARDT: return x2_kernel<T, N, MODE_REACT, BCT, SFRD_REACT_GIERER_MEINHARDT>;
        case SFRD_REACT_LINEAR: return x2_kernel<T, N, MODE_REACT, BCT, SFRD_REACT_LINEAR>;
        default: return x2_kernel<T, N, MODE_REACT, BCT, SFRD_REACT_NONE>;
    }
}

template <typename T, int N, int BCT>
cudaError_t x2_launch_bc(const XArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    const size_t smem = TileOf<T, N>::E::smem_bytes();
    void (*k)(const XArgs<T>) =
        mode == MODE_REACT ? x2_kernel<T, N, MODE_REACT, BCT> : x2_kernel<T, N, MODE_PLAIN, BCT>;
    if constexpr (KindSpecialised<T, N>::value) {
        if (mode == MODE_REACT && a.S == 2 && !a.save) k = x2_kind_kernel<T, N, BCT>(a.re.kind);
    }
    k<<<grid, kThreads, smem, s>>>(a);
    return cudaGetLastError();
}

template <typename T, int N, int BCT>
cudaError_t x2_prepare_bc() {
    void (*xs[])(const XArgs<T>) = {x2_kernel<T, N, MODE_PLAIN, BCT>, x2_kernel<T, N, MODE_REACT, BCT>};
    for (auto k : xs) {
        const cudaError_t e = set_smem_attrs(k, kMaxDynSmem2);
        if (e != cudaSuccess) return e;
    }
    if constexpr (KindSpecialised<T, N>::value) {
        const int kinds[] = {SFRD_REACT_NONE, SFRD_REACT_LINEAR, SFRD_REACT_FHN, SFRD_REACT_GRAY_SCOTT,
                             SFRD_REACT_SCHNAKENBERG, SFRD_REACT_GIERER_MEINHARDT};
        for (int kind : kinds) {
            const cudaError_t e = set_smem_attrs(x2_kind_kernel<T, N, BCT>(kind), kMaxDynSmem2);
            if (e != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}

// Column-pass dispatch to the family (instantiates no kernel itself).
template <typename T, int N, int BCT>
cudaError_t col2_launch_bc(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    if constexpr (sizeof(T) == 4) {
        if (is_stage_mode(mode) && a.cstride == 2 && a.in_sp > 0) return col2_pair_launch_bc<T, N, BCT>(a, mode, grid, s);
        if (is_stage_mode(mode) && a.CL) return col2_rat_launch_bc<T, N, BCT>(a, mode, grid, s);
    }
    return col2_plain_launch_bc<T, N, BCT>(a, mode, grid, s);
}

template <typename T, int N, int BCT>
cudaError_t prepare2_bc() {
    cudaError_t e = col2_plain_prepare_bc<T, N, BCT>();
    if (e == cudaSuccess) e = col2_pair_prepare_bc<T, N, BCT>();
    if (e == cudaSuccess) e = col2_rat_prepare_bc<T, N, BCT>();
    if (e == cudaSuccess) e = x2_prepare_bc<T, N, BCT>();
    return e;
}

template <typename T, int N>
cudaError_t col2_launch(const ColArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    if constexpr (BcSpecialised<T, N>::value) {
        switch (a.ax.bc) {
            case SFRD_BC_PERIODIC: return col2_launch_bc<T, N, SFRD_BC_PERIODIC>(a, mode, grid, s);
            case SFRD_BC_DIRICHLET: return col2_launch_bc<T, N, SFRD_BC_DIRICHLET>(a, mode, grid, s);
            default: return col2_launch_bc<T, N, SFRD_BC_NEUMANN>(a, mode, grid, s);
        }
    }
    return col2_launch_bc<T, N, -1>(a, mode, grid, s);
}

template <typename T, int N>
cudaError_t x2_launch(const XArgs<T>& a, int mode, dim3 grid, cudaStream_t s) {
    if constexpr (BcSpecialised<T, N>::value) {
        switch (a.ax.bc) {
            case SFRD_BC_PERIODIC: return x2_launch_bc<T, N, SFRD_BC_PERIODIC>(a, mode, grid, s);
            case SFRD_BC_DIRICHLET: return x2_launch_bc<T, N, SFRD_BC_DIRICHLET>(a, mode, grid, s);
            default: return x2_launch_bc<T, N, SFRD_BC_NEUMANN>(a, mode, grid, s);
        }
    }
    return x2_launch_bc<T, N, -1>(a, mode, grid, s);
}

template <typename T, int N>
cudaError_t prepare2() {
    if constexpr (BcSpecialised<T, N>::value) {
        cudaError_t e = prepare2_bc<T, N, SFRD_BC_PERIODIC>();
        if (e == cudaSuccess) e = prepare2_bc<T, N, SFRD_BC_DIRICHLET>();
        if (e == cudaSuccess) e = prepare2_bc<T, N, SFRD_BC_NEUMANN>();
        if (e != cudaSuccess) return e;
    }
    return prepare2_bc<T, N, -1>();
}

// Explicit instantiation.  SFRD_V2_INSTANTIATE emits a whole length in one object; a length split over
// several objects emits SFRD_V2_DISPATCH once and each family macro in an object of its own.  The
// dispatchers are only declared where they are not emitted.
#define SFRD_V2_DISPATCH_BC(T, N, BCT)                                                             \
    template cudaError_t col2_launch_bc<T, N, BCT>(const ColArgs<T>&, int, dim3, cudaStream_t);   \
    template cudaError_t prepare2_bc<T, N, BCT>();

#define SFRD_V2_DISPATCH(T, N)                                                                     \
    template cudaError_t col2_launch<T, N>(const ColArgs<T>&, int, dim3, cudaStream_t);           \
    template cudaError_t x2_launch<T, N>(const XArgs<T>&, int, dim3, cudaStream_t);               \
    template cudaError_t prepare2<T, N>();                                                        \
    SFRD_V2_DISPATCH_BC(T, N, -1)

#define SFRD_V2_PLAIN(T, N, BCT)                                                                   \
    template cudaError_t col2_plain_launch_bc<T, N, BCT>(const ColArgs<T>&, int, dim3, cudaStream_t); \
    template cudaError_t col2_plain_prepare_bc<T, N, BCT>();

#define SFRD_V2_PAIR(T, N, BCT)                                                                    \
    template cudaError_t col2_pair_launch_bc<T, N, BCT>(const ColArgs<T>&, int, dim3, cudaStream_t); \
    template cudaError_t col2_pair_prepare_bc<T, N, BCT>();

#define SFRD_V2_RAT(T, N, BCT)                                                                     \
    template cudaError_t col2_rat_launch_bc<T, N, BCT>(const ColArgs<T>&, int, dim3, cudaStream_t); \
    template cudaError_t col2_rat_prepare_bc<T, N, BCT>();

#define SFRD_V2_X(T, N, BCT)                                                                       \
    template cudaError_t x2_launch_bc<T, N, BCT>(const XArgs<T>&, int, dim3, cudaStream_t);       \
    template cudaError_t x2_prepare_bc<T, N, BCT>();

// Declares the families of a split length as instantiated elsewhere (keeps the dispatch object free of kernels).
#define SFRD_V2_EXTERN_FAMILIES(T, N, BCT)                                                                  \
    extern template cudaError_t col2_plain_launch_bc<T, N, BCT>(const ColArgs<T>&, int, dim3, cudaStream_t); \
    extern template cudaError_t col2_plain_prepare_bc<T, N, BCT>();                                         \
    extern template cudaError_t col2_pair_launch_bc<T, N, BCT>(const ColArgs<T>&, int, dim3, cudaStream_t);  \
    extern template cudaError_t col2_pair_prepare_bc<T, N, BCT>();                                          \
    extern template cudaError_t col2_rat_launch_bc<T, N, BCT>(const ColArgs<T>&, int, dim3, cudaStream_t);   \
    extern template cudaError_t col2_rat_prepare_bc<T, N, BCT>();                                           \
    extern template cudaError_t x2_launch_bc<T, N, BCT>(const XArgs<T>&, int, dim3, cudaStream_t);          \
    extern template cudaError_t x2_prepare_bc<T, N, BCT>();

#define SFRD_V2_INSTANTIATE_BC(T, N, BCT)                                                          \
    SFRD_V2_DISPATCH_BC(T, N, BCT)                                                                 \
    SFRD_V2_PLAIN(T, N, BCT)                                                                       \
    SFRD_V2_PAIR(T, N, BCT)                                                                        \
    SFRD_V2_RAT(T, N, BCT)                                                                         \
    SFRD_V2_X(T, N, BCT)

#define SFRD_V2_INSTANTIATE(T, N)                                                                  \
    template cudaError_t col2_launch<T, N>(const ColArgs<T>&, int, dim3, cudaStream_t);           \
    template cudaError_t x2_launch<T, N>(const XArgs<T>&, int, dim3, cudaStream_t);               \
    template cudaError_t prepare2<T, N>();                                                        \
    SFRD_V2_INSTANTIATE_BC(T, N, -1)

}  // namespace v2
}  // namespace sfrd
