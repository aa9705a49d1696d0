// Shared-memory column FFT engine.
//
// A tile is a block of CC complex columns of length M held in shared memory as
// buf[row * ldb + col].  Two real lines are packed into one complex column
// (real part = line A, imaginary part = line B), so every real transform of the
// solver -- the discrete Hartley transform for periodic axes, DST-I for
// Dirichlet and DCT-I for Neumann (Section 3.1: the eigenvector matrices of
// Eqs. PP, PD, PN) -- is obtained from one forward complex DFT of length M
// (M = N, or M = 2N on the odd/even extension of the line, the construction
// the paper takes from its reference for Eq. PN) followed by an O(M) unpacking.
//
// Thread (grp, c): c = column (lane within a group of CC threads), grp = one of
// G = blockDim / CC groups that share the butterflies of a stage.  All lanes of
// a group work on the same butterfly, so twiddle and permutation loads are
// uniform and shared-memory accesses are consecutive words.
//
// The DFT is computed in place, mixed radix (2, 3, 4, 5, 8):
//   DIF: natural-order input  -> output in slot perm[k];
//   DIT (radices reversed): input taken from slot perm[n] -> natural-order output.
// A barrier separates stages; each thread owns the R slots of its butterfly.
#pragma once

#include "sfrd_internal.h"

namespace sfrd {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename C> __device__ __forceinline__ C mul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }  // * (-i)
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
template <typename C> __device__ __forceinline__ C cneg(C a) { C r; r.x = -a.x; r.y = -a.y; return r; }
template <typename C> __device__ __forceinline__ C czero() { C r; r.x = 0; r.y = 0; return r; }
// a * s + b for a real s
template <typename C, typename T> __device__ __forceinline__ C cfma(C a, T s, C b) {
    C r; r.x = a.x * s + b.x; r.y = a.y * s + b.y; return r;
}

// FP32 complex values use the paired single-precision instructions of sm_100 and later
// (both halves of a 64-bit register pair in one instruction, each rounded as the scalar
// operation would be).
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(rd));
    return r;
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 cfma(float2 a, float s, float2 b) { return __ffma2_rn(a, make_float2(s, s), b); }

template <typename C> __device__ __forceinline__ C ldtw(const C* tw, int i) { return __ldg(tw + i); }

// ---- small DFTs, forward sign exp(-2 pi i r m / R), in registers ----------------

template <int R, typename C> struct Dft;

template <typename C> struct Dft<2, C> {
    static __device__ __forceinline__ void run(C* a) { C t = a[0]; a[0] = cadd(t, a[1]); a[1] = csub(t, a[1]); }
};

template <typename C> struct Dft<4, C> {
    static __device__ __forceinline__ void run(C* a) {
        C t0 = cadd(a[0], a[2]), t1 = csub(a[0], a[2]);
        C t2 = cadd(a[1], a[3]), t3 = mul_mi(csub(a[1], a[3]));
        a[0] = cadd(t0, t2); a[2] = csub(t0, t2);
        a[1] = cadd(t1, t3); a[3] = csub(t1, t3);
    }
};

template <typename C> struct Dft<8, C> {
    static __device__ __forceinline__ void run(C* a) {
        using T = decltype(a[0].x);
        const T c = (T)0.70710678118654752440;   // 1/sqrt(2)
        C e[4] = {a[0], a[2], a[4], a[6]};
        C o[4] = {a[1], a[3], a[5], a[7]};
        Dft<4, C>::run(e);
        Dft<4, C>::run(o);
        C o1, o3;
        o1.x = c * (o[1].x + o[1].y); o1.y = c * (o[1].y - o[1].x);    // * exp(-i pi/4)
        C o2 = mul_mi(o[2]);                                              // * exp(-i pi/2)
        o3.x = c * (o[3].y - o[3].x); o3.y = -c * (o[3].x + o[3].y);   // * exp(-3 i pi/4)
        a[0] = cadd(e[0], o[0]); a[4] = csub(e[0], o[0]);
        a[1] = cadd(e[1], o1);   a[5] = csub(e[1], o1);
        a[2] = cadd(e[2], o2);   a[6] = csub(e[2], o2);
        a[3] = cadd(e[3], o3);   a[7] = csub(e[3], o3);
    }
};

template <typename C> struct Dft<3, C> {
    static __device__ __forceinline__ void run(C* a) {
        using T = decltype(a[0].x);
        const T s3 = (T)0.86602540378443864676;   // sin(2 pi / 3)
        C s = cadd(a[1], a[2]), d = csub(a[1], a[2]);
        C t; t.x = a[0].x - (T)0.5 * s.x; t.y = a[0].y - (T)0.5 * s.y;
        C r; r.x = s3 * d.y; r.y = -s3 * d.x;     // -i sin(2pi/3) d
        a[0] = cadd(a[0], s);
        a[1] = cadd(t, r);
        a[2] = csub(t, r);
    }
};

template <typename C> struct Dft<5, C> {
    static __device__ __forceinline__ void run(C* a) {
        using T = decltype(a[0].x);
        const T c1 = (T)0.30901699437494742410;    // cos(2 pi / 5)
        const T c2 = (T)-0.80901699437494742410;   // cos(4 pi / 5)
        const T s1 = (T)0.95105651629515357212;    // sin(2 pi / 5)
        const T s2 = (T)0.58778525229247312917;    // sin(4 pi / 5)
        C b1 = cadd(a[1], a[4]), b2 = cadd(a[2], a[3]);
        C d1 = csub(a[1], a[4]), d2 = csub(a[2], a[3]);
        C t1, t2, u1, u2;
        t1.x = a[0].x + c1 * b1.x + c2 * b2.x; t1.y = a[0].y + c1 * b1.y + c2 * b2.y;
        t2.x = a[0].x + c2 * b1.x + c1 * b2.x; t2.y = a[0].y + c2 * b1.y + c1 * b2.y;
        u1.x = s1 * d1.x + s2 * d2.x; u1.y = s1 * d1.y + s2 * d2.y;
        u2.x = s2 * d1.x - s1 * d2.x; u2.y = s2 * d1.y - s1 * d2.y;
        a[0] = cadd(a[0], cadd(b1, b2));
        C m1 = mul_mi(u1), m2 = mul_mi(u2);
        a[1] = cadd(t1, m1); a[4] = csub(t1, m1);
        a[2] = cadd(t2, m2); a[3] = csub(t2, m2);
    }
};

// ---- one in-place stage ---------------------------------------------------------

// DIF stage on blocks of length L (stride s = L/R): y = DFT_R(x); y_m *= omega_L^{j m}.
template <int R, typename C>
__device__ __forceinline__ void dif_stage(C* buf, int ldb, int M, int L, const C* __restrict__ tw,
                                          int c, int grp, int G) {
    const int s = L / R, nb = M / R, twstep = M / L;
    for (int b = grp; b < nb; b += G) {
        const int g = b / s, j = b - g * s;
        const int base = g * L + j;
        C a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = buf[(base + r * s) * ldb + c];
        Dft<R, C>::run(a);
        if (j != 0) {
#pragma unroll
            for (int m = 1; m < R; ++m) a[m] = cmul(a[m], ldtw(tw, j * m * twstep));
        }
#pragma unroll
        for (int m = 0; m < R; ++m) buf[(base + m * s) * ldb + c] = a[m];
    }
}

// DIT stage combining R sub-transforms of length Lp: x_r *= omega_L^{j r}; y = DFT_R(x).
template <int R, typename C>
__device__ __forceinline__ void dit_stage(C* buf, int ldb, int M, int Lp, const C* __restrict__ tw,
                                          int c, int grp, int G) {
    const int L = Lp * R, nb = M / R, twstep = M / L;
    for (int b = grp; b < nb; b += G) {
        const int g = b / Lp, j = b - g * Lp;
        const int base = g * L + j;
        C a[R];
#pragma unroll
        for (int r = 0; r < R; ++r) a[r] = buf[(base + r * Lp) * ldb + c];
        if (j != 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) a[r] = cmul(a[r], ldtw(tw, j * r * twstep));
        }
        Dft<R, C>::run(a);
#pragma unroll
        for (int m = 0; m < R; ++m) buf[(base + m * Lp) * ldb + c] = a[m];
    }
}

// Forward DFT, natural order in, slot perm[k] out.  Ends with a barrier.
template <typename C>
__device__ void fft_dif(C* buf, int ldb, const AxisDev& ax, int c, int grp, int G) {
    const C* tw = static_cast<const C*>(ax.tw);
    int L = ax.M;
    for (int t = 0; t < ax.nst; ++t) {
        const int R = ax.radix[t];
        switch (R) {
            case 8: dif_stage<8>(buf, ldb, ax.M, L, tw, c, grp, G); break;
            case 4: dif_stage<4>(buf, ldb, ax.M, L, tw, c, grp, G); break;
            case 2: dif_stage<2>(buf, ldb, ax.M, L, tw, c, grp, G); break;
            case 3: dif_stage<3>(buf, ldb, ax.M, L, tw, c, grp, G); break;
            default: dif_stage<5>(buf, ldb, ax.M, L, tw, c, grp, G); break;
        }
        L /= R;
        __syncthreads();
    }
}

// Forward DFT, input in slot perm[n], natural order out.  Ends with a barrier.
template <typename C>
__device__ void fft_dit(C* buf, int ldb, const AxisDev& ax, int c, int grp, int G) {
    const C* tw = static_cast<const C*>(ax.tw);
    int Lp = 1;
    for (int t = ax.nst - 1; t >= 0; --t) {
        const int R = ax.radix[t];
        switch (R) {
            case 8: dit_stage<8>(buf, ldb, ax.M, Lp, tw, c, grp, G); break;
            case 4: dit_stage<4>(buf, ldb, ax.M, Lp, tw, c, grp, G); break;
            case 2: dit_stage<2>(buf, ldb, ax.M, Lp, tw, c, grp, G); break;
            case 3: dit_stage<3>(buf, ldb, ax.M, Lp, tw, c, grp, G); break;
            default: dit_stage<5>(buf, ldb, ax.M, Lp, tw, c, grp, G); break;
        }
        Lp *= R;
        __syncthreads();
    }
}

// ---- packing of real lines into the complex FFT input ---------------------------
//
// Unknown i of the line (0 <= i < n) sits at extension index
//   periodic: i;  Dirichlet: i + 1 (mirror 2N - 1 - i with sign -1, zeros at 0 and N);
//   Neumann: i (mirror 2N - i for 0 < i < N).
// `slot` maps an extension index to its buffer row.

__device__ __forceinline__ int ext_index(int bc, int i) { return bc == SFRD_BC_DIRICHLET ? i + 1 : i; }

// Writes the value z of unknown i and its mirror.  slot: identity (natural) or perm.
template <typename C, bool PERM>
__device__ __forceinline__ void put_extended(C* buf, int ldb, const AxisDev& ax, int i, int c, C z) {
    const int e = ext_index(ax.bc, i);
    const int r0 = PERM ? __ldg(ax.perm + e) : e;
    buf[r0 * ldb + c] = z;
    if (ax.bc == SFRD_BC_DIRICHLET) {
        const int e2 = 2 * ax.N - e;
        const int r1 = PERM ? __ldg(ax.perm + e2) : e2;
        buf[r1 * ldb + c] = cneg(z);
    } else if (ax.bc == SFRD_BC_NEUMANN && e > 0 && e < ax.N) {
        const int e2 = 2 * ax.N - e;
        const int r1 = PERM ? __ldg(ax.perm + e2) : e2;
        buf[r1 * ldb + c] = z;
    }
}

// Zeros of the odd extension (Dirichlet only), written by group 0.
template <typename C, bool PERM>
__device__ __forceinline__ void put_extension_zeros(C* buf, int ldb, const AxisDev& ax, int c, int grp) {
    if (ax.bc == SFRD_BC_DIRICHLET && grp == 0) {
        const int r0 = PERM ? __ldg(ax.perm + 0) : 0;
        const int r1 = PERM ? __ldg(ax.perm + ax.N) : ax.N;
        buf[r0 * ldb + c] = czero<C>();
        buf[r1 * ldb + c] = czero<C>();
    }
}

// Number of work items of the unpacking step: one per unknown (Dirichlet,
// Neumann) or one per Hartley pair {k, N-k} (periodic).
__device__ __forceinline__ int unpack_items(const AxisDev& ax) {
    return ax.bc == SFRD_BC_PERIODIC ? ax.N / 2 + 1 : ax.n;
}

// Reads the transform of lines A and B at item `it` from the DFT output.
// Returns 1 or 2 outputs (k0, k1); (A0,B0) at k0, (A1,B1) at k1.
template <typename C, bool PERM>
__device__ __forceinline__ int get_transform(const C* buf, int ldb, const AxisDev& ax, int it, int c,
                                             int& k0, C& v0, int& k1, C& v1) {
    using T = decltype(v0.x);
    if (ax.bc == SFRD_BC_PERIODIC) {
        const int N = ax.N;
        k0 = it;
        k1 = (N - it) % N;
        const int r0 = PERM ? __ldg(ax.perm + k0) : k0;
        const int r1 = PERM ? __ldg(ax.perm + k1) : k1;
        const C z0 = buf[r0 * ldb + c], z1 = buf[r1 * ldb + c];
        // Hartley: H_A = (p_k + p_-k + q_-k - q_k)/2, H_B = (q_k + q_-k + p_k - p_-k)/2
        v0.x = (T)0.5 * (z0.x + z1.x + z1.y - z0.y);
        v0.y = (T)0.5 * (z0.y + z1.y + z0.x - z1.x);
        v1.x = (T)0.5 * (z1.x + z0.x + z0.y - z1.y);
        v1.y = (T)0.5 * (z1.y + z0.y + z1.x - z0.x);
        return (k1 == k0) ? 1 : 2;
    }
    k0 = it;
    const int e = ext_index(ax.bc, it);
    const int r0 = PERM ? __ldg(ax.perm + e) : e;
    const C z = buf[r0 * ldb + c];
    if (ax.bc == SFRD_BC_DIRICHLET) {   // DST-I: A = -Im Z / 2, B = Re Z / 2
        v0.x = (T)-0.5 * z.y;
        v0.y = (T)0.5 * z.x;
    } else {                            // DCT-I: A = Re Z / 2, B = Im Z / 2
        v0.x = (T)0.5 * z.x;
        v0.y = (T)0.5 * z.y;
    }
    return 1;
}

// Writes the new value of unknown k (of item it) as the next transform's input.
template <typename C, bool PERM>
__device__ __forceinline__ void put_value(C* buf, int ldb, const AxisDev& ax, int k, int c, C z) {
    if (ax.bc == SFRD_BC_PERIODIC) {
        const int r0 = PERM ? __ldg(ax.perm + k) : k;
        buf[r0 * ldb + c] = z;
    } else {
        put_extended<C, PERM>(buf, ldb, ax, k, c, z);
    }
}

}  // namespace sfrd
