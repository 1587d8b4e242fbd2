// In-place FFT engine with two transforms per thread in packed FP32x2
// registers.
//
// The transform is the DFT of Sec. 2.3 Eq. (10) (0-based indices, forward
// sign -, unnormalised both ways), factored N = R_0 R_1 ... R_{S-1} by
// Cooley-Tukey (Sec. 2.3 cites the FFT's N log N cost).  Here the forward
// transform runs decimation in frequency (DIF) in place and leaves the
// spectrum in digit-reversed position order; the inverse runs decimation in
// time (DIT) in place, the forward's stages transposed in reverse order, so
// it takes exactly that order and returns natural order.  The map never
// needs the spectrum in natural order except where a pass stores it (the
// row pass's half spectra) or loads it (the inverse row pass), and there a
// position table maps frequencies to positions.
//
// Stage s of a length-N transform, with B_s = N / (R_0 ... R_{s-1}) (block
// size) and D_s = B_s / R_s (stride): butterfly (blk, j), blk < N / B_s,
// j < D_s, owns the R_s elements at blk B_s + j + m D_s.
//   forward (DIF):  y_k = sum_m x_m exp(-i 2 pi m k / R_s),
//                   y_k *= exp(-i 2 pi j k / B_s), stored at index k
//   inverse (DIT):  x_k *= exp(+i 2 pi j k / B_s),
//                   y_m = sum_k x_k exp(+i 2 pi m k / R_s), stored at index m
// After all forward stages, position p = sum_s k_s D_s holds the frequency
// f = k_0 + R_0 (k_1 + R_1 (k_2 + ...)).  The last stage has D = 1, so the
// butterfly blk of the last stage holds the frequencies
//   f(blk) + k N / R_{S-1},  k < R_{S-1}:
// the forward's last stage, the spectrum product and the inverse's first
// stage run on the same registers.
//
// Every stage is in place, so a butterfly reads and writes only its own
// elements: one barrier per stage, and a thread processes its butterflies
// one after another (registers do not grow with the butterflies per thread).
//
// Two transforms per thread.  A value of type CP holds element n of two
// independent transforms A and B as {re A, re B}, {im A, im B}; every
// complex operation of the DFT is then one packed FP32x2 instruction per
// component (add.f32x2 / mul.f32x2 / fma.f32x2), the same instruction
// stream serving both transforms.  The single-transform type float2 {re, im}
// serves lengths whose two-transform buffer does not fit shared memory.
#pragma once

#include "fft_core.cuh"
#include "lp_internal.h"

namespace lpk {

// ---------------------------------------------------------------------------
// packed FP32x2 arithmetic
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 pk(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}
// sign flip by integer xor (integer pipe, exact)
__device__ __forceinline__ float2 neg2(float2 a)
{
    return make_float2(__int_as_float(__float_as_int(a.x) ^ 0x80000000),
                       __int_as_float(__float_as_int(a.y) ^ 0x80000000));
}

// element n of two transforms: x = {re A, re B}, y = {im A, im B}
struct CP {
    float2 x, y;
};

// ---------------------------------------------------------------------------
// complex operations on one value (float2) or on a pair (CP)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return add2(a, b); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return sub2(a, b); }
__device__ __forceinline__ float2 c_scale(float2 a, float c) { return mul2(a, pk(c)); }
__device__ __forceinline__ float2 c_fma(float2 a, float c, float2 acc) { return fma2(a, pk(c), acc); }
__device__ __forceinline__ float2 c_neg(float2 a) { return neg2(a); }
// a + DIR i b
template <int DIR>
__device__ __forceinline__ float2 c_addi(float2 a, float2 b)
{
    return DIR > 0 ? make_float2(a.x - b.y, a.y + b.x) : make_float2(a.x + b.y, a.y - b.x);
}
// D i a (D = +-1)
template <int D>
__device__ __forceinline__ float2 c_muli(float2 a)
{
    return D > 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}
// a * (c + i s), c and s constants
__device__ __forceinline__ float2 c_rotc(float2 a, float c, float s)
{
    return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}

__device__ __forceinline__ CP c_add(CP a, CP b) { return CP{add2(a.x, b.x), add2(a.y, b.y)}; }
__device__ __forceinline__ CP c_sub(CP a, CP b) { return CP{sub2(a.x, b.x), sub2(a.y, b.y)}; }
__device__ __forceinline__ CP c_scale(CP a, float c) { return CP{mul2(a.x, pk(c)), mul2(a.y, pk(c))}; }
__device__ __forceinline__ CP c_fma(CP a, float c, CP acc) { return CP{fma2(a.x, pk(c), acc.x), fma2(a.y, pk(c), acc.y)}; }
__device__ __forceinline__ CP c_neg(CP a) { return CP{neg2(a.x), neg2(a.y)}; }
template <int DIR>
__device__ __forceinline__ CP c_addi(CP a, CP b)
{
    return DIR > 0 ? CP{sub2(a.x, b.y), add2(a.y, b.x)} : CP{add2(a.x, b.y), sub2(a.y, b.x)};
}
template <int D>
__device__ __forceinline__ CP c_muli(CP a)
{
    return D > 0 ? CP{neg2(a.y), a.x} : CP{a.y, neg2(a.x)};
}
__device__ __forceinline__ CP c_rotc(CP a, float c, float s)
{
    return CP{fma2(a.y, pk(-s), mul2(a.x, pk(c))), fma2(a.y, pk(c), mul2(a.x, pk(s)))};
}

// a * exp(DIR i 2 pi T / N), T and N compile-time
template <int T, int N, int DIR, class C>
__device__ __forceinline__ C c_rot(C a)
{
    constexpr int t = ((T % N) + N) % N;
    if constexpr (t == 0) {
        return a;
    } else if constexpr (2 * t == N) {
        return c_neg(a);
    } else if constexpr (4 * t == N || 4 * t == 3 * N) {
        return c_muli<(4 * t == N) ? DIR : -DIR>(a);
    } else {
        return c_rotc(a, (float)cos2pi(t, N), (float)(DIR * sin2pi(t, N)));
    }
}

// ---------------------------------------------------------------------------
// In-register DFT of size R (unnormalised, natural order in and out), for
// C = float2 or CP.  Radix 2 and 4 by hand; odd primes by the symmetric pair
// formula; composites with coprime factors by the prime-factor mapping (no
// internal twiddles); other composites by Cooley-Tukey with constant
// rotations.
// ---------------------------------------------------------------------------
template <int R, int DIR, class C> struct D2;

template <int DIR, class C> struct D2<1, DIR, C> {
    __device__ __forceinline__ static void run(C*) {}
};

template <int DIR, class C> struct D2<2, DIR, C> {
    __device__ __forceinline__ static void run(C* v)
    {
        const C a = v[0], b = v[1];
        v[0] = c_add(a, b);
        v[1] = c_sub(a, b);
    }
};

template <int DIR, class C> struct D2<4, DIR, C> {
    __device__ __forceinline__ static void run(C* v)
    {
        const C t0 = c_add(v[0], v[2]), t1 = c_sub(v[0], v[2]);
        const C t2 = c_add(v[1], v[3]), t3 = c_sub(v[1], v[3]);
        v[0] = c_add(t0, t2);
        v[2] = c_sub(t0, t2);
        v[1] = c_addi<DIR>(t1, t3);
        v[3] = c_addi<-DIR>(t1, t3);
    }
};

// odd prime P: with a_k = x_k + x_{P-k}, b_k = x_k - x_{P-k},
// y_m = x_0 + sum_k a_k cos(2 pi k m / P) + DIR i sum_k b_k sin(2 pi k m / P)
// and y_{P-m} the same with -DIR
template <int P, int DIR, class C>
__device__ __forceinline__ void d2_odd_prime(C* v)
{
    constexpr int H = (P - 1) / 2;
    C a[H], b[H];
    sfor<1, H + 1>([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        a[k - 1] = c_add(v[k], v[P - k]);
        b[k - 1] = c_sub(v[k], v[P - k]);
    });
    C y[P];
    y[0] = v[0];
    sfor<0, H>([&](auto K_) { y[0] = c_add(y[0], a[decltype(K_)::value]); });
    sfor<1, H + 1>([&](auto M_) {
        constexpr int m = decltype(M_)::value;
        C re = v[0];
        C im;
        sfor<1, H + 1>([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            constexpr float c = (float)cos2pi((long)k * m, P);
            constexpr float s = (float)sin2pi((long)k * m, P);
            re = c_fma(a[k - 1], c, re);
            im = (k == 1) ? c_scale(b[0], s) : c_fma(b[k - 1], s, im);
        });
        y[m] = c_addi<DIR>(re, im);
        y[P - m] = c_addi<-DIR>(re, im);
    });
    sfor<0, P>([&](auto K_) { v[decltype(K_)::value] = y[decltype(K_)::value]; });
}

template <int R, int DIR, class C> struct D2 {
    static constexpr int A = small_factor(R);
    static constexpr int B = R / A;
    __device__ __forceinline__ static void run(C* v)
    {
        if constexpr (A == 1) {
            static_assert(R % 2 == 1, "prime radix must be odd here");
            d2_odd_prime<R, DIR, C>(v);
        } else if constexpr (gcd_i(A, B) == 1) {
            // prime-factor mapping: n = (B n1 + A n2) mod R, k = CRT(k1, k2)
            constexpr int EA = B * inv_mod(B % A, A);
            constexpr int EB = A * inv_mod(A % B, B);
            C t[R];
            sfor<0, B>([&](auto N2_) {
                constexpr int n2 = decltype(N2_)::value;
                C a[A];
                sfor<0, A>([&](auto N1_) {
                    constexpr int n1 = decltype(N1_)::value;
                    a[n1] = v[(B * n1 + A * n2) % R];
                });
                D2<A, DIR, C>::run(a);
                sfor<0, A>([&](auto K1_) { t[n2 * A + decltype(K1_)::value] = a[decltype(K1_)::value]; });
            });
            sfor<0, A>([&](auto K1_) {
                constexpr int k1 = decltype(K1_)::value;
                C b[B];
                sfor<0, B>([&](auto N2_) { b[decltype(N2_)::value] = t[decltype(N2_)::value * A + k1]; });
                D2<B, DIR, C>::run(b);
                sfor<0, B>([&](auto K2_) {
                    constexpr int k2 = decltype(K2_)::value;
                    v[(k1 * EA + k2 * EB) % R] = b[k2];
                });
            });
        } else {
            // Cooley-Tukey: n = B n1 + n2, k = k1 + A k2
            C t[R];
            sfor<0, B>([&](auto N2_) {
                constexpr int n2 = decltype(N2_)::value;
                C a[A];
                sfor<0, A>([&](auto N1_) { a[decltype(N1_)::value] = v[B * decltype(N1_)::value + n2]; });
                D2<A, DIR, C>::run(a);
                sfor<0, A>([&](auto K1_) {
                    constexpr int k1 = decltype(K1_)::value;
                    t[n2 * A + k1] = c_rot<n2 * k1, R, DIR>(a[k1]);
                });
            });
            sfor<0, A>([&](auto K1_) {
                constexpr int k1 = decltype(K1_)::value;
                C b[B];
                sfor<0, B>([&](auto N2_) { b[decltype(N2_)::value] = t[decltype(N2_)::value * A + k1]; });
                D2<B, DIR, C>::run(b);
                sfor<0, B>([&](auto K2_) { v[k1 + A * decltype(K2_)::value] = b[decltype(K2_)::value]; });
            });
        }
    }
};

// ---------------------------------------------------------------------------
// Twiddles.  One table per length, W[i] = exp(-i 2 pi i / N), i < N, as
// {cos, sin} (TwTab2::w).  Stage s needs exp(-i 2 pi j k / B_s) =
// W[(j k N / B_s) mod N]; the exponent of k is k times that of k = 1, so it is
// stepped by one addition and a conditional subtraction.  All stages and all
// blocks of an SM share the one table, which stays in L1.
// ---------------------------------------------------------------------------
// v *= w (DIR < 0, the forward twiddle) or v *= conj(w) (DIR > 0)
template <int DIR>
__device__ __forceinline__ void tw_apply(CP& v, float2 w)
{
    const float2 wr = pk(w.x);
    const float2 wi = pk(DIR < 0 ? w.y : -w.y);
    const float2 nwi = pk(DIR < 0 ? -w.y : w.y);
    const CP r{fma2(v.y, nwi, mul2(v.x, wr)), fma2(v.x, wi, mul2(v.y, wr))};
    v = r;
}
template <int DIR>
__device__ __forceinline__ void tw_apply(float2& v, float2 w)
{
    const float c = w.x, s = DIR < 0 ? w.y : -w.y;
    v = make_float2(v.x * c - v.y * s, v.x * s + v.y * c);
}

// the R-1 twiddles of butterfly j of a stage with block size Bs, applied to
// v[1..R-1]; the loads are issued first, all together
template <int N, int R, int Bs, int DIR, class C>
__device__ __forceinline__ void twiddle_all(C (&v)[R], int j, const float2* __restrict__ W)
{
    constexpr int STEP = N / Bs;
    const int e1 = j * STEP;  // < N / R_s
    float2 w[R - 1];
    int e = 0;
#pragma unroll
    for (int k = 1; k < R; ++k) {
        e += e1;
        if (e >= N) e -= N;
        w[k - 1] = __ldg(W + e);
    }
#pragma unroll
    for (int k = 1; k < R; ++k) tw_apply<DIR>(v[k], w[k - 1]);
}

// ---------------------------------------------------------------------------
// Geometry of a plan: radices R_0..R_{S-1} in forward (DIF) order.
// ---------------------------------------------------------------------------
template <int N, int... Rs>
struct IpGeom {
    static constexpr int S = sizeof...(Rs);
    static constexpr int r(int s)
    {
        const int rs[] = {Rs...};
        return rs[s];
    }
    static constexpr int B(int s)  // block size of stage s
    {
        int b = N;
        for (int i = 0; i < s; ++i) b /= r(i);
        return b;
    }
    static constexpr int D(int s) { return B(s) / r(s); }  // stride of stage s
    static constexpr int RL = r(S - 1);
    static constexpr int R0 = r(0);
    // butterflies of stage s visited with consecutive j (else consecutive blk):
    // consecutive threads then touch consecutive 16-byte elements, or
    // elements B_s apart (conflict-free when B_s is odd)
    static constexpr bool jfast(int s) { return D(s) >= 8 || (B(s) % 2 == 0 && D(s) > 1); }
};

// base index of butterfly b of stage s
template <class G, int s>
__device__ __forceinline__ int ip_base(int b, int& j)
{
    constexpr int Bs = G::B(s), Ds = G::D(s), NBLK = (G::B(0)) / Bs;
    if constexpr (G::jfast(s)) {
        j = b % Ds;
        return (b / Ds) * Bs + j;
    } else {
        j = b / NBLK;
        return (b % NBLK) * Bs + j;
    }
}

// One in-place stage over the elements X[0..N) of shared memory, T threads.
// FWD: DIF (DFT then twiddle); else DIT (conjugate twiddle then DFT).
template <class G, int s, bool FWD, int T, class C>
__device__ __forceinline__ void ip_stage(C* X, int t, const TwTab2& tw)
{
    constexpr int R = G::r(s), Ds = G::D(s), NB = G::B(0) / R;
    constexpr int E = (NB + T - 1) / T;
#pragma unroll 1
    for (int e = 0; e < E; ++e) {
        const int b = t + e * T;
        if (NB % T != 0 && b >= NB) break;
        int j;
        const int base = ip_base<G, s>(b, j);
        C v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = X[base + k * Ds];
        if constexpr (!FWD && Ds > 1) twiddle_all<G::B(0), R, G::B(s), +1>(v, j, tw.w);
        D2<R, FWD ? -1 : +1, C>::run(v);
        if constexpr (FWD && Ds > 1) twiddle_all<G::B(0), R, G::B(s), -1>(v, j, tw.w);
#pragma unroll
        for (int k = 0; k < R; ++k) X[base + k * Ds] = v[k];
    }
}

// Forward stages [s0, s1) with a barrier after each.
template <class G, int s0, int s1, int T, class C>
__device__ __forceinline__ void ip_forward(C* X, int t, const TwTab2& tw)
{
    if constexpr (s0 < s1) {
        ip_stage<G, s0, true, T, C>(X, t, tw);
        __syncthreads();
        ip_forward<G, s0 + 1, s1, T, C>(X, t, tw);
    }
}
// Inverse stages s1-1 down to s0 with a barrier after each.
template <class G, int s0, int s1, int T, class C>
__device__ __forceinline__ void ip_inverse(C* X, int t, const TwTab2& tw)
{
    if constexpr (s0 < s1) {
        ip_stage<G, s1 - 1, false, T, C>(X, t, tw);
        __syncthreads();
        ip_inverse<G, s0, s1 - 1, T, C>(X, t, tw);
    }
}

// Stage 0 of the forward transform with the inputs from a loader
// (ld(index) returns element `index` of the zero-padded input) and the
// outputs to shared memory.
template <class G, int T, class C, class Ld>
__device__ __forceinline__ void ip_first_forward(C* X, int t, const TwTab2& tw, Ld&& ld)
{
    constexpr int R = G::R0, Ds = G::D(0), NB = G::B(0) / R;
    constexpr int E = (NB + T - 1) / T;
    static_assert(G::jfast(0) || Ds == 1, "stage 0 visits consecutive j");
#pragma unroll 1
    for (int e = 0; e < E; ++e) {
        const int b = t + e * T;
        if (NB % T != 0 && b >= NB) break;
        const int j = b;  // one block in stage 0
        C v[R];
#pragma unroll
        for (int m = 0; m < R; ++m) v[m] = ld(j + m * Ds);
        D2<R, -1, C>::run(v);
        if constexpr (Ds > 1) twiddle_all<G::B(0), R, G::B(0), -1>(v, j, tw.w);
#pragma unroll
        for (int k = 0; k < R; ++k) X[j + k * Ds] = v[k];
    }
}

// Stage 0 of the inverse transform from shared memory, outputs to a sink
// (st(index, value), index = natural-order output index).
template <class G, int T, class C, class St>
__device__ __forceinline__ void ip_last_inverse(const C* X, int t, const TwTab2& tw, St&& st)
{
    constexpr int R = G::R0, Ds = G::D(0), NB = G::B(0) / R;
    constexpr int E = (NB + T - 1) / T;
#pragma unroll 1
    for (int e = 0; e < E; ++e) {
        const int b = t + e * T;
        if (NB % T != 0 && b >= NB) break;
        const int j = b;
        C v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = X[j + k * Ds];
        if constexpr (Ds > 1) twiddle_all<G::B(0), R, G::B(0), +1>(v, j, tw.w);
        D2<R, +1, C>::run(v);
#pragma unroll
        for (int m = 0; m < R; ++m) st(j + m * Ds, v[m]);
    }
}

// The forward's last stage, a per-element operation, and the inverse's
// first stage on the same registers: op(p, v) is applied to the value v at
// position p (the frequency held there is given by the position table).
template <class G, int T, class C, class Op>
__device__ __forceinline__ void ip_middle(C* X, int t, Op&& op)
{
    constexpr int R = G::RL, NB = G::B(0) / R;
    constexpr int E = (NB + T - 1) / T;
#pragma unroll 1
    for (int e = 0; e < E; ++e) {
        const int blk = t + e * T;
        if (NB % T != 0 && blk >= NB) break;
        C v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = X[blk * R + k];
        D2<R, -1, C>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) op(blk * R + k, v[k]);
        D2<R, +1, C>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) X[blk * R + k] = v[k];
    }
}

// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (the transform's input staged in
// shared memory with every load in flight at once; cp.async.wait_group is a
// hardware wait)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cpa16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cpa_wait_all()
{
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

}  // namespace lpk
