// Register FFT engine for the axis lengths N with an in-register split N = R1 x R2 (Split<N>):
// the powers of two 16..1024 and 96, 200, 384.
//
// Each real transform of the solver (Section 3.1: Hartley for periodic axes,
// DST-I for Dirichlet, DCT-I for Neumann) is computed from ONE complex FFT of
// length N carrying two real lines (real part = line A, imaginary part = B):
//
//   periodic:  z_j = x_j;                                    T_k = R_k + I_k, T_{N-k} = R_k - I_k
//   Dirichlet: z_j = s_j (x_j + x_{N-j}) + (x_j - x_{N-j})/2 T_{2k} = I_k,  T_{2k+1} = T_{2k-1} + R_k
//   Neumann:   z_j = (x_j + x_{N-j})/2 - s_j (x_j - x_{N-j}) T_{2k} = R_k,  T_{2k+1} = T_{2k-1} + I_k
// with s_j = sin(j pi / N), x the line on grid nodes (x_0 = x_N = 0 for
// Dirichlet), and R_k - i I_k the DFT of the pre-processed real line, unpacked
// from the packed complex DFT.  The odd-index outputs of DST-I / DCT-I follow
// from a running sum, done as a two-level prefix sum over the half spectrum;
// its anchor is T_1 = R_0 / 2 (Dirichlet) or T_1 = (x_0 - x_N)/2 +
// sum_j x_j cos(j pi / N) (Neumann).  These are the classical real-FFT
// pre/post-processings of the sine and cosine transforms: pairing j with N-j
// splits the kernel sin(pi j k'/N) (or cos) into the even part, a plain real
// DFT, and the odd part, whose products with s_j telescope in k'.
//
// The complex FFT is a two-step decomposition N = R1 x R2 entirely in
// registers (j = R2 n1 + n2, k = k1 + R1 k2): step 1 owns n2 and does a
// DFT-R1 over n1 followed by the twiddles omega_N^{n2 k1}; one shared-memory
// exchange; step 2 owns k1 and does a DFT-R2 over n2, writing X in natural
// order into the same slots it read.  All sizes and loop bounds are
// compile-time constants.
//
// Tile: CC columns (lane c), G = 256 / CC groups (g).  Shared memory holds one
// buffer of max(n, N) rows x (CC + 1) complex: it is the value buffer V (row =
// unknown index) before the pre-processing and after the post-processing, and
// the FFT buffer Z in between; barriers separate the two uses.
#pragma once

#include <type_traits>

#include "engine.cuh"

namespace sfrd {
namespace v2 {

// ---- compile-time trigonometry (Taylor series on a reduced argument) -------------

constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double ce_sin_small(double x) {
    double x2 = x * x, t = x, s = x;
    for (int i = 1; i < 16; ++i) {
        t *= -x2 / ((2.0 * i) * (2.0 * i + 1.0));
        s += t;
    }
    return s;
}

constexpr double ce_cos_small(double x) {
    double x2 = x * x, t = 1.0, s = 1.0;
    for (int i = 1; i < 16; ++i) {
        t *= -x2 / ((2.0 * i - 1.0) * (2.0 * i));
        s += t;
    }
    return s;
}

struct CS {
    double c, s;
};

// cos and sin of 2 pi m / R, argument reduced exactly on the integers.
constexpr CS ce_cs2pi(long m, long R) {
    long r = m % R;
    if (r < 0) r += R;
    const long q = (4 * r) / R;
    const long rem = 4 * r - q * R;
    double c0 = 0, s0 = 0;
    if (2 * rem <= R) {
        const double ph = (kPi / 2) * (double)rem / (double)R;
        c0 = ce_cos_small(ph);
        s0 = ce_sin_small(ph);
    } else {
        const double ph = (kPi / 2) * (double)(R - rem) / (double)R;
        c0 = ce_sin_small(ph);
        s0 = ce_cos_small(ph);
    }
    switch (q) {
        case 0: return CS{c0, s0};
        case 1: return CS{-s0, c0};
        case 2: return CS{-c0, -s0};
        default: return CS{s0, -c0};
    }
}

// a * omega_R^M, omega_R = exp(-2 pi i / R), M and R compile-time constants (quarter turns as
// exchanges and sign changes when 4 divides R).
template <int M, int R, typename C> __device__ __forceinline__ C mul_wr(C a) {
    using T = decltype(a.x);
    constexpr int m = ((M % R) + R) % R;
    if constexpr (m == 0) {
        return a;
    } else if constexpr (R % 4 == 0 && m == R / 4) {
        return mul_mi(a);
    } else if constexpr (R % 2 == 0 && m == R / 2) {
        return cneg(a);
    } else if constexpr (R % 4 == 0 && m == 3 * R / 4) {
        C r; r.x = -a.y; r.y = a.x; return r;
    } else {
        constexpr T wr = (T)ce_cs2pi(m, R).c, wi = (T)(-ce_cs2pi(m, R).s);
        C r; r.x = a.x * wr - a.y * wi; r.y = a.x * wi + a.y * wr; return r;
    }
}

// Compile-time loop: f(std::integral_constant<int, i>) for i = B .. E-1.
template <int B, int E, class F> __device__ __forceinline__ void static_for(F&& f) {
    if constexpr (B < E) {
        f(std::integral_constant<int, B>());
        static_for<B + 1, E>(f);
    }
}

// ---- in-register DFTs of length 2..32 (natural order in and out) -----------------

template <int R, typename C> struct RDft {
    static __device__ __forceinline__ void run(C* a) { Dft<R, C>::run(a); }
};

// R = Ra * Rb four-step: j = Rb j1 + j2, k = k1 + Ra k2.
template <int R, int Ra, typename C> struct FourStep {
    static constexpr int Rb = R / Ra;
    static __device__ __forceinline__ void run(C* a) {
        C t[R];
        static_for<0, Rb>([&](auto J2) {
            constexpr int j2 = decltype(J2)::value;
            C u[Ra];
#pragma unroll
            for (int j1 = 0; j1 < Ra; ++j1) u[j1] = a[Rb * j1 + j2];
            RDft<Ra, C>::run(u);
            static_for<0, Ra>([&](auto K1) {
                constexpr int k1 = decltype(K1)::value;
                t[j2 * Ra + k1] = mul_wr<j2 * k1, R>(u[k1]);
            });
        });
#pragma unroll
        for (int k1 = 0; k1 < Ra; ++k1) {
            C w[Rb];
#pragma unroll
            for (int j2 = 0; j2 < Rb; ++j2) w[j2] = t[j2 * Ra + k1];
            RDft<Rb, C>::run(w);
#pragma unroll
            for (int k2 = 0; k2 < Rb; ++k2) a[k1 + Ra * k2] = w[k2];
        }
    }
};

template <typename C> struct RDft<16, C> {
    static __device__ __forceinline__ void run(C* a) { FourStep<16, 4, C>::run(a); }
};
template <typename C> struct RDft<32, C> {
    static __device__ __forceinline__ void run(C* a) { FourStep<32, 8, C>::run(a); }
};
// composite lengths with factors 3 and 5 (the non-power-of-two axis lengths of the engine)
template <typename C> struct RDft<6, C> {
    static __device__ __forceinline__ void run(C* a) { FourStep<6, 2, C>::run(a); }
};
template <typename C> struct RDft<10, C> {
    static __device__ __forceinline__ void run(C* a) { FourStep<10, 2, C>::run(a); }
};
template <typename C> struct RDft<12, C> {
    static __device__ __forceinline__ void run(C* a) { FourStep<12, 4, C>::run(a); }
};
template <typename C> struct RDft<20, C> {
    static __device__ __forceinline__ void run(C* a) { FourStep<20, 4, C>::run(a); }
};
template <typename C> struct RDft<24, C> {
    static __device__ __forceinline__ void run(C* a) { FourStep<24, 8, C>::run(a); }
};

// ---- the line engine ----------------------------------------------------------------

template <int N> struct Split;
template <> struct Split<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct Split<32> { static constexpr int R1 = 4, R2 = 8; };
template <> struct Split<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Split<128> { static constexpr int R1 = 8, R2 = 16; };
template <> struct Split<256> { static constexpr int R1 = 16, R2 = 16; };
template <> struct Split<512> { static constexpr int R1 = 16, R2 = 32; };
template <> struct Split<1024> { static constexpr int R1 = 32, R2 = 32; };
// 3 * 2^5, 5^2 * 2^3 and 3 * 2^7 (the Gierer-Meinhardt batch's other sides)
template <> struct Split<96> { static constexpr int R1 = 6, R2 = 16; };
template <> struct Split<200> { static constexpr int R1 = 10, R2 = 20; };
template <> struct Split<384> { static constexpr int R1 = 16, R2 = 24; };

// Columns per tile for a power-of-two axis length.
template <typename T, int N> struct TileCC { static constexpr int value = cc_for(sizeof(T) == 8, N); };

// BCT: the boundary condition as a compile-time constant (SFRD_BC_*), or -1 when it is
// taken from the runtime argument.
template <typename T, int N, int CC, int BCT = -1>
struct Eng {
    static __device__ __forceinline__ int bcv(int bc) { return BCT >= 0 ? BCT : bc; }
    using C = typename Cx<T>::type;
    static constexpr int G = kThreads / CC;
    static constexpr int R1 = Split<N>::R1, R2 = Split<N>::R2;
    static constexpr int LD = CC + 1;
    static constexpr int H = N / 2;
    static constexpr int CH = (H + G - 1) / G;      // half-spectrum pairs per group
    static constexpr int NO1 = (R2 + G - 1) / G;    // step-1 owners per thread
    static constexpr int NO2 = (R1 + G - 1) / G;    // step-2 owners per thread
    static constexpr int ROWS = N + 1;              // buffer rows (n <= N + 1)

    static constexpr size_t smem_bytes() {
        return (size_t)ROWS * LD * sizeof(C) + (size_t)2 * G * CC * sizeof(C) + (size_t)2 * N * sizeof(C);
    }

    // Pre-processed input z_j of the packed DFT, read from the value buffer.
    static __device__ __forceinline__ C pre(const C* V, int bc_, int j, int c, const C* tws, C& anchor) {
        return pre_w(V, bc_, j, c, tws[j], anchor);
    }

    // The same with w = (cos(j pi/N), -sin(j pi/N)) given.
    static __device__ __forceinline__ C pre_w(const C* V, int bc_, int j, int c, C w, C& anchor) {
        const int bc = bcv(bc_);
        if (bc == SFRD_BC_PERIODIC) return V[j * LD + c];
        const T s = -w.y;
        if (bc == SFRD_BC_DIRICHLET) {
            if (j == 0) return czero<C>();
            const C xj = V[(j - 1) * LD + c], xm = V[(N - j - 1) * LD + c];
            return cfma(cadd(xj, xm), s, cscale(csub(xj, xm), (T)0.5));
        }
        const C xj = V[j * LD + c], xm = V[(N - j) * LD + c];
        const C dif = csub(xj, xm);
        if (j == 0) anchor = cfma(dif, (T)0.5, anchor);
        else anchor = cfma(xj, w.x, anchor);
        return cfma(dif, -s, cscale(cadd(xj, xm), (T)0.5));
    }

    // Pre-processing of a mirror pair: z_j and z_{N-j} from the line's values xj, xm at transform
    // indices j and N - j (x_0 = x_N = 0 for Dirichlet; xm unused for periodic), with s = sin(j pi/N) and
    // co = cos(j pi/N); the Neumann anchor gains this pair's share (x_j - x_{N-j}) cos(j pi/N), or
    // (x_0 - x_N)/2 for j = 0.  One thread then writes both, so every value is read once.
    static __device__ __forceinline__ void pre_pair(int bc_, int j, C xj, C xm, T s, T co, C& zj, C& zm, C& anchor) {
        const int bc = bcv(bc_);
        if (bc == SFRD_BC_PERIODIC) {
            zj = xj;
            zm = xm;
            return;
        }
        const C sum = cadd(xj, xm), dif = csub(xj, xm);
        if (bc == SFRD_BC_DIRICHLET) {
            const C o = cscale(dif, (T)0.5);
            zj = cfma(sum, s, o);
            zm = cfma(sum, s, cneg(o));
            return;
        }
        const C e = cscale(sum, (T)0.5);
        zj = cfma(dif, -s, e);
        zm = cfma(dif, s, e);
        anchor = j == 0 ? cfma(dif, (T)0.5, anchor) : cfma(dif, co, anchor);
    }

    // forward() for a buffer that already holds the pre-processed line z (natural order, written with
    // pre_pair) and red2 the Neumann anchor parts.  Entry: z complete (after a barrier).
    static __device__ __forceinline__ void forward_z(C* buf, int bc_, const C* tws, int twstride_, int c, int g) {
        forward_impl<true>(buf, nullptr, bc_, tws, twstride_, c, g);
    }

    // V (natural, unknown index) -> pre-processing -> DFT_N -> Z (natural order).
    // Entry: V complete (after a barrier).  Exit: Z complete (after a barrier).
    // red2[g][c] receives this thread's part of the Neumann anchor.
    // tws: the axis table in shared memory, omega_{N*twstride}^m (twstride = 1 periodic, 2 otherwise).
    static __device__ __forceinline__ void forward(C* buf, C* red2, int bc_, const C* tws, int twstride_, int c,
                                                   int g) {
        forward_impl<false>(buf, red2, bc_, tws, twstride_, c, g);
    }

    // ZIN: the buffer holds z already (forward_z); else the values V, pre-processed on the way in.
    template <bool ZIN>
    static __device__ __forceinline__ void forward_impl(C* buf, C* red2, int bc_, const C* tws, int twstride_, int c,
                                                        int g) {
        const int bc = bcv(bc_);
        const int twstride = BCT < 0 ? twstride_ : (BCT == SFRD_BC_PERIODIC ? 1 : 2);
        C a[NO1][R1];
        C anchor = czero<C>();
#pragma unroll
        for (int o = 0; o < NO1; ++o) {
            const int n2 = g + o * G;
            if (R2 % G == 0 || n2 < R2) {
                if constexpr (ZIN) {
#pragma unroll
                    for (int n1 = 0; n1 < R1; ++n1) a[o][n1] = buf[(R2 * n1 + n2) * LD + c];
                } else {
                    // w_j for j = R2 n1 + n2 by rotating w_{n2} (one table read) through the
                    // compile-time angle R2 n1 pi / N
                    const C wb = bc == SFRD_BC_PERIODIC ? czero<C>() : tws[n2];
                    static_for<0, R1>([&](auto N1) {
                        constexpr int n1 = decltype(N1)::value;
                        constexpr T cr = (T)ce_cs2pi(R2 * n1, 2 * N).c, ci = (T)(-ce_cs2pi(R2 * n1, 2 * N).s);
                        C w;
                        w.x = wb.x * cr - wb.y * ci;
                        w.y = wb.x * ci + wb.y * cr;
                        a[o][n1] = pre_w(buf, bc, R2 * n1 + n2, c, w, anchor);
                    });
                }
                RDft<R1, C>::run(a[o]);
                if (R1 <= 16) {
                    // omega_N^{n2 k1} = (omega_N^{4 n2})^{k1 / 4} (omega_N^{n2})^{k1 % 4}: two table reads
                    constexpr int NQ = (R1 + 3) / 4;
                    C pw[4], qw[NQ > 1 ? NQ : 2];
                    pw[1] = tws[n2 * twstride];
                    pw[2] = cmul(pw[1], pw[1]);
                    pw[3] = cmul(pw[2], pw[1]);
                    if (NQ > 1) qw[1] = tws[4 * n2 * twstride];
                    if (NQ > 2) qw[2] = cmul(qw[1], qw[1]);
                    if (NQ > 3) qw[3] = cmul(qw[2], qw[1]);
#pragma unroll
                    for (int k1 = 1; k1 < R1; ++k1) {
                        const int qq = k1 / 4, r = k1 % 4;
                        if (qq > 0) a[o][k1] = cmul(a[o][k1], qw[qq]);
                        if (r > 0) a[o][k1] = cmul(a[o][k1], pw[r]);
                    }
                } else {
#pragma unroll
                    for (int k1 = 1; k1 < R1; ++k1) a[o][k1] = cmul(a[o][k1], tws[(n2 * k1) * twstride]);
                }
            }
        }
        if constexpr (!ZIN) red2[g * CC + c] = anchor;
        __syncthreads();   // all reads of V done: the buffer becomes Z
#pragma unroll
        for (int o = 0; o < NO1; ++o) {
            const int n2 = g + o * G;
            if (R2 % G == 0 || n2 < R2) {
#pragma unroll
                for (int k1 = 0; k1 < R1; ++k1) buf[(n2 * R1 + k1) * LD + c] = a[o][k1];
            }
        }
        __syncthreads();
#pragma unroll
        for (int o = 0; o < NO2; ++o) {
            const int k1 = g + o * G;
            if (R1 % G == 0 || k1 < R1) {
                C b[R2];
#pragma unroll
                for (int n2 = 0; n2 < R2; ++n2) b[n2] = buf[(n2 * R1 + k1) * LD + c];
                RDft<R2, C>::run(b);
#pragma unroll
                for (int k2 = 0; k2 < R2; ++k2) buf[(k1 + R1 * k2) * LD + c] = b[k2];
            }
        }
        __syncthreads();
    }

    // Z (natural) -> transform values; sink(i, value) is called for every unknown i
    // of this thread's output range after a barrier (so the sink may write V).
    // Emission in batches of B half-spectrum pairs: pre(slot, i) is called for every output i
    // of a batch before sink(slot, i, value) is called for them, so that a caller can issue
    // all global loads of a batch together (slot < 2B is a compile-time index).
    template <int B, class Pre, class Sink>
    static __device__ __forceinline__ void post_b(C* buf, C* red, const C* red2, int bc_, int c, int g, Pre&& pre,
                                                  Sink&& sink) {
        const int bc = bcv(bc_);
        C ev[CH], od[CH];   // even-index outputs, running odd-index partial sums
        C run = czero<C>();
        const int k0 = g * CH;
#pragma unroll
        for (int t = 0; t < CH; ++t) {
            const int k = k0 + t;
            if (k < H) {
                const C zk = buf[k * LD + c];
                const C zm = buf[((N & (N - 1)) == 0 ? ((N - k) & (N - 1)) : (k == 0 ? 0 : N - k)) * LD + c];
                const C Rk = cscale(cadd(zk, zm), (T)0.5);
                const C d = csub(zk, zm);
                C Ik;
                Ik.x = (T)-0.5 * d.y;
                Ik.y = (T)0.5 * d.x;
                if (bc == SFRD_BC_PERIODIC) {
                    ev[t] = cadd(Rk, Ik);     // T_k
                    od[t] = csub(Rk, Ik);     // T_{N-k}
                } else if (bc == SFRD_BC_DIRICHLET) {
                    ev[t] = Ik;
                    C d = Rk;
                    if (k == 0) { d.x *= (T)0.5; d.y *= (T)0.5; }
                    run = cadd(run, d);
                    od[t] = run;
                } else {
                    ev[t] = Rk;
                    C d = Ik;
                    if (k == 0) {
                        d = czero<C>();
#pragma unroll 4
                        for (int q = 0; q < G; ++q) d = cadd(d, red2[q * CC + c]);
                    }
                    run = cadd(run, d);
                    od[t] = run;
                }
            }
        }
        C nyq = czero<C>();
        if (bc != SFRD_BC_DIRICHLET && g == G - 1) {
            const C zh = buf[H * LD + c];     // k = N/2: R = Re, I = 0 for both lines
            nyq = zh;
        }
        // running sums of the groups before this one (same column): within the warp by an exclusive
        // shuffle scan over its 32 / CC groups, across warps from the per-warp column totals in red
        static_assert(32 % CC == 0, "a warp holds whole groups");
        constexpr int GPW = 32 / CC;           // groups per warp
        const int w = g / GPW, lane = (g % GPW) * CC + c;
        C pre_sum = czero<C>();
        if (bc != SFRD_BC_PERIODIC) {
            if (GPW > 1) {
                C ex;                          // the shifted sequence: running sum of the previous group
                ex.x = __shfl_up_sync(0xffffffffu, run.x, CC);
                ex.y = __shfl_up_sync(0xffffffffu, run.y, CC);
                if (lane < CC) ex = czero<C>();
#pragma unroll
                for (int d = CC; d < 32 - CC; d *= 2) {
                    C t;
                    t.x = __shfl_up_sync(0xffffffffu, ex.x, d);
                    t.y = __shfl_up_sync(0xffffffffu, ex.y, d);
                    if (lane >= d) ex = cadd(ex, t);
                }
                pre_sum = ex;
            }
            if (lane >= 32 - CC) red[w * CC + c] = cadd(pre_sum, run);
        }
        __syncthreads();   // all reads of Z done: the buffer becomes V
        if (bc != SFRD_BC_PERIODIC) {
            for (int q = 0; q < w; ++q) pre_sum = cadd(pre_sum, red[q * CC + c]);
        }
        // output q (0, 1) of pair t: index and value, or false when there is none
        auto out_of = [&](int t, int q, int& i, C& v) -> bool {
            const int k = k0 + t;
            if (k >= H) return false;
            if (bc == SFRD_BC_PERIODIC) {
                if (q == 0) { i = k; v = ev[t]; return true; }
                if (k == 0) return false;
                i = N - k; v = od[t]; return true;
            }
            if (bc == SFRD_BC_DIRICHLET) {
                if (q == 0) {
                    if (k == 0) return false;
                    i = 2 * k - 1; v = ev[t]; return true;
                }
                i = 2 * k; v = cadd(pre_sum, od[t]); return true;
            }
            if (q == 0) { i = 2 * k; v = ev[t]; return true; }
            i = 2 * k + 1; v = cadd(pre_sum, od[t]); return true;
        };
#pragma unroll
        for (int t0 = 0; t0 < CH; t0 += B) {
#pragma unroll
            for (int t = t0; t < t0 + B && t < CH; ++t) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    int i;
                    C v;
                    if (out_of(t, q, i, v)) pre(2 * (t - t0) + q, i);
                }
            }
#pragma unroll
            for (int t = t0; t < t0 + B && t < CH; ++t) {
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    int i;
                    C v;
                    if (out_of(t, q, i, v)) sink(2 * (t - t0) + q, i, v);
                }
            }
        }
        if (bc != SFRD_BC_DIRICHLET && g == G - 1) {
            const int i = bc == SFRD_BC_PERIODIC ? H : N;
            pre(0, i);
            sink(0, i, nyq);
        }
    }

    template <class Sink>
    static __device__ __forceinline__ void post(C* buf, C* red, const C* red2, int bc, int c, int g, Sink&& sink) {
        post_b<CH>(buf, red, red2, bc, c, g, [](int, int) {}, [&](int, int i, C v) { sink(i, v); });
    }
};

}  // namespace v2
}  // namespace sfrd
