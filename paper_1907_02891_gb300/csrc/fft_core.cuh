// Device building blocks of the FFT path: compile-time trigonometry,
// in-register DFTs of small radices, and Stockham stage chains that exchange
// data through padded structure-of-arrays shared memory.
//
// The transform computed is the DFT of Sec. 2.3 Eq. (10) (0-based indices),
// F[k] = sum_n f[n] exp(DIR * i 2 pi k n / N), DIR = -1 forward, +1 inverse
// (unnormalised both ways), evaluated by the Cooley-Tukey factorisation the
// paper cites for FFTs (Sec. 2.3): N = R_0 R_1 ... R_{S-1}, one radix-R_s
// butterfly stage per factor, in the self-sorting (Stockham) arrangement so
// that the output comes out in natural order without a bit-reversal pass.
//
// Stage s of a chain, with Ns = R_0 ... R_{s-1} and butterfly index
// j in [0, N/R_s):
//   inputs   x[j + m N/R_s],                      m = 0..R_s-1
//   twiddle  x_m *= exp(DIR i 2 pi (j mod Ns) m / (Ns R_s))
//   DFT of size R_s in registers
//   outputs  y[(j div Ns) Ns R_s + (j mod Ns) + m Ns]
// In the last stage Ns = N / R_{S-1}, so thread j holds y[j + m N/R_{S-1}]:
// exactly the set the first stage of a chain with the same radix reads.  The
// convolution kernels use that to multiply by the PSF spectrum between the
// forward and the inverse column transform without touching shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "lp_internal.h"

namespace lpk {

// ---------------------------------------------------------------------------
// Compile-time trigonometry: cos / sin of 2 pi t / n for integer t, n.
// The angle is reduced to a quadrant in exact integer arithmetic, then a
// Taylor series in double precision (16 terms on |x| <= pi/4, truncation far
// below 1e-17) is summed.  Only used to build constants at compile time.
// ---------------------------------------------------------------------------
constexpr double kHalfPi = 1.57079632679489661923132169163975;

__host__ __device__ constexpr double taylor_sin(double x)
{
    double term = x, sum = x;
    for (int k = 1; k < 16; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

__host__ __device__ constexpr double taylor_cos(double x)
{
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 16; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// cos(phi), sin(phi) for phi = (pi/2) r / n, 0 <= r < n, with the argument
// kept in [0, pi/4] by the complementary-angle identity.
__host__ __device__ constexpr double quad_cos(long r, long n)
{
    return (2 * r <= n) ? taylor_cos(kHalfPi * (double)r / (double)n)
                        : taylor_sin(kHalfPi * (double)(n - r) / (double)n);
}
__host__ __device__ constexpr double quad_sin(long r, long n)
{
    return (2 * r <= n) ? taylor_sin(kHalfPi * (double)r / (double)n)
                        : taylor_cos(kHalfPi * (double)(n - r) / (double)n);
}

__host__ __device__ constexpr double cos2pi(long t, long n)
{
    t = ((t % n) + n) % n;
    const long q = (4 * t) / n, r = 4 * t - q * n;
    const double c = quad_cos(r, n), s = quad_sin(r, n);
    return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
__host__ __device__ constexpr double sin2pi(long t, long n)
{
    t = ((t % n) + n) % n;
    const long q = (4 * t) / n, r = 4 * t - q * n;
    const double c = quad_cos(r, n), s = quad_sin(r, n);
    return q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
}

// ---------------------------------------------------------------------------
// Compile-time loop helper: calls f(integral_constant<int, I>) for I in [B, E).
// ---------------------------------------------------------------------------
template <int B, int E, class F>
__device__ __forceinline__ void sfor(F&& f)
{
    if constexpr (B < E) {
        f(std::integral_constant<int, B>{});
        sfor<B + 1, E>(f);
    }
}

// ---------------------------------------------------------------------------
// Complex helpers, generic over float2 / double2.
// ---------------------------------------------------------------------------
template <class C> struct Scalar;
template <> struct Scalar<float2> { using type = float; };
template <> struct Scalar<double2> { using type = double; };

template <class C>
__device__ __forceinline__ C mk(typename Scalar<C>::type x, typename Scalar<C>::type y)
{
    C r;
    r.x = x;
    r.y = y;
    return r;
}
template <class C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
// a * c (c real) and a * c + acc
template <class C> __device__ __forceinline__ C cscale(C a, typename Scalar<C>::type c)
{
    return mk<C>(a.x * c, a.y * c);
}
template <class C> __device__ __forceinline__ C cfma(C a, typename Scalar<C>::type c, C acc)
{
    return mk<C>(a.x * c + acc.x, a.y * c + acc.y);
}

// FP32 complex values {re, im} are a natural pair for the packed FP32x2
// instructions: an addition, a subtraction, a real scaling or a real
// multiply-add of a complex value is one add / sub / mul / fma .f32x2.
// A plan chooses per length (LP_PACKED_FP32, set by the length's translation
// unit, whose device code is compiled on its own): the packed constants take
// registers, which costs more than it saves in the register-bound kernels of
// some lengths.
#ifndef LP_PACKED_FP32
#define LP_PACKED_FP32 1
#endif
#if LP_PACKED_FP32
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b)
{
    unsigned long long ra, rb, rd;
    asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
    asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
    float2 d;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
    return d;
}
__device__ __forceinline__ float2 cscale(float2 a, float c) { return __fmul2_rn(a, make_float2(c, c)); }
__device__ __forceinline__ float2 cfma(float2 a, float c, float2 acc) { return __ffma2_rn(a, make_float2(c, c), acc); }
#endif
template <class C> __device__ __forceinline__ C cmul(C a, C b)
{
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// multiply by i*DIR (DIR = +-1)
template <int DIR, class C> __device__ __forceinline__ C mul_idir(C a)
{
    if constexpr (DIR > 0) return mk<C>(-a.y, a.x);
    else return mk<C>(a.y, -a.x);
}

// a * exp(DIR i 2 pi t / n), with t, n compile-time.  Exact quarter turns are
// done by swaps, eighth turns with one shared factor, the rest by a complex
// multiply against rounded constants.
template <int T, int N, int DIR, class C>
__device__ __forceinline__ C rot(C a)
{
    using S = typename Scalar<C>::type;
    constexpr int t = ((T % N) + N) % N;
    if constexpr (t == 0) {
        return a;
    } else if constexpr (2 * t == N) {
        return mk<C>(-a.x, -a.y);
    } else if constexpr (4 * t == N) {
        return mul_idir<DIR>(a);
    } else if constexpr (4 * t == 3 * N) {
        return mul_idir<-DIR>(a);
    } else if constexpr ((8 * t) % N == 0) {
        // odd multiple of an eighth turn: cos, sin = +-sqrt(1/2)
        constexpr S h = (S)0.70710678118654752440084436210485;
        constexpr S cs = (S)(cos2pi(t, N) > 0 ? 1 : -1);
        constexpr S sn = (S)((sin2pi(t, N) > 0 ? 1 : -1) * DIR);
        // (x + i y)(cs + i sn) h
        return mk<C>(h * (cs * a.x - sn * a.y), h * (sn * a.x + cs * a.y));
    } else {
        constexpr S c = (S)cos2pi(t, N);
        constexpr S s = (S)(DIR * sin2pi(t, N));
        return mk<C>(a.x * c - a.y * s, a.x * s + a.y * c);
    }
}

// ---------------------------------------------------------------------------
// In-register DFT of size R (unnormalised), natural order in and out.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int gcd_i(int a, int b) { return b == 0 ? a : gcd_i(b, a % b); }

// Split of a composite radix r = a * b for the in-register DFT: coprime
// factors when there are any (prime-factor algorithm, no internal
// twiddles), the largest such a with a*a <= r; otherwise the largest
// divisor a with a*a <= r (4 x r/4 for powers of two).  1 for primes.
__host__ __device__ constexpr int small_factor(int r)
{
    int coprime = 1;
    for (int a = 2; a < r; ++a)
        if (r % a == 0 && gcd_i(a, r / a) == 1 && (coprime == 1 || a * a <= r)) coprime = a;
    if (coprime > 1) {
        // prefer the smaller of the two coprime factors first
        const int b = r / coprime;
        return coprime < b ? coprime : b;
    }
    if (r % 4 == 0 && r > 4) return 4;
    int best = 1;
    for (int a = 2; a * a <= r; ++a)
        if (r % a == 0) best = a;
    return best;
}

// modular inverse of a mod m (a, m coprime), compile time
__host__ __device__ constexpr int inv_mod(int a, int m)
{
    for (int x = 1; x < m; ++x)
        if ((a * x) % m == 1) return x;
    return 1;
}

template <int R, int DIR, class C> struct Dft;

template <int DIR, class C> struct Dft<1, DIR, C> {
    __device__ __forceinline__ static void run(C*) {}
};

template <int DIR, class C> struct Dft<2, DIR, C> {
    __device__ __forceinline__ static void run(C* v)
    {
        C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    }
};

template <int DIR, class C> struct Dft<4, DIR, C> {
    __device__ __forceinline__ static void run(C* v)
    {
        C t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        C t2 = cadd(v[1], v[3]), t3 = mul_idir<DIR>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2);
        v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3);
        v[3] = csub(t1, t3);
    }
};

// Odd prime P: pair x_k with x_{P-k}; y_m = x_0 + sum_k (x_k + x_{P-k}) cos
// + DIR i sum_k (x_k - x_{P-k}) sin, and y_{P-m} the conjugate combination.
template <int P, int DIR, class C>
__device__ __forceinline__ void dft_odd_prime(C* v)
{
    using S = typename Scalar<C>::type;
    constexpr int H = (P - 1) / 2;
    C a[H], b[H];
    sfor<1, H + 1>([&](auto K_) {
        constexpr int k = decltype(K_)::value;
        a[k - 1] = cadd(v[k], v[P - k]);
        b[k - 1] = csub(v[k], v[P - k]);
    });
    C y[P];
    y[0] = v[0];
    sfor<0, H>([&](auto K_) { y[0] = cadd(y[0], a[decltype(K_)::value]); });
    sfor<1, H + 1>([&](auto M_) {
        constexpr int m = decltype(M_)::value;
        C re = v[0];
        C im;
        sfor<1, H + 1>([&](auto K_) {
            constexpr int k = decltype(K_)::value;
            constexpr S c = (S)cos2pi((long)k * m, P);
            constexpr S s = (S)sin2pi((long)k * m, P);
            re = cfma(a[k - 1], c, re);
            im = (k == 1) ? cscale(b[0], s) : cfma(b[k - 1], s, im);
        });
        // y_m = re + DIR i im ; y_{P-m} = re - DIR i im
        C ii = mul_idir<DIR>(im);
        y[m] = cadd(re, ii);
        y[P - m] = csub(re, ii);
    });
    sfor<0, P>([&](auto K_) { v[decltype(K_)::value] = y[decltype(K_)::value]; });
}

// Composite R = A * B.
//  * gcd(A, B) = 1: prime-factor (Good-Thomas) algorithm.  With input index
//    n = (B n1 + A n2) mod R and output index k = k1 B (B^-1 mod A) +
//    k2 A (A^-1 mod B) mod R (k1 = k mod A, k2 = k mod B), the R-point DFT
//    is A-point DFTs over n1 followed by B-point DFTs over n2 with no
//    twiddles in between; both index maps are compile-time permutations.
//  * otherwise Cooley-Tukey in registers: n = B n1 + n2, k = k1 + A k2;
//    A-point DFTs over n1, twiddle exp(DIR i 2pi n2 k1 / R), B-point DFTs
//    over n2.
template <int R, int DIR, class C> struct Dft {
    static constexpr int A = small_factor(R);
    static constexpr int B = R / A;
    __device__ __forceinline__ static void run(C* v)
    {
        if constexpr (A == 1) {
            static_assert(R % 2 == 1, "prime radix must be odd here");
            dft_odd_prime<R, DIR, C>(v);
        } else if constexpr (gcd_i(A, B) == 1) {
            constexpr int EA = B * inv_mod(B % A, A);  // k -> k1 component of the CRT
            constexpr int EB = A * inv_mod(A % B, B);
            C t[R];
            sfor<0, B>([&](auto N2_) {
                constexpr int n2 = decltype(N2_)::value;
                C a[A];
                sfor<0, A>([&](auto N1_) {
                    constexpr int n1 = decltype(N1_)::value;
                    a[n1] = v[(B * n1 + A * n2) % R];
                });
                Dft<A, DIR, C>::run(a);
                sfor<0, A>([&](auto K1_) { t[n2 * A + decltype(K1_)::value] = a[decltype(K1_)::value]; });
            });
            sfor<0, A>([&](auto K1_) {
                constexpr int k1 = decltype(K1_)::value;
                C b[B];
                sfor<0, B>([&](auto N2_) { b[decltype(N2_)::value] = t[decltype(N2_)::value * A + k1]; });
                Dft<B, DIR, C>::run(b);
                sfor<0, B>([&](auto K2_) {
                    constexpr int k2 = decltype(K2_)::value;
                    v[(k1 * EA + k2 * EB) % R] = b[k2];
                });
            });
        } else {
            C t[R];
            sfor<0, B>([&](auto N2_) {
                constexpr int n2 = decltype(N2_)::value;
                C a[A];
                sfor<0, A>([&](auto N1_) { a[decltype(N1_)::value] = v[B * decltype(N1_)::value + n2]; });
                Dft<A, DIR, C>::run(a);
                sfor<0, A>([&](auto K1_) {
                    constexpr int k1 = decltype(K1_)::value;
                    t[n2 * A + k1] = rot<n2 * k1, R, DIR>(a[k1]);
                });
            });
            sfor<0, A>([&](auto K1_) {
                constexpr int k1 = decltype(K1_)::value;
                C b[B];
                sfor<0, B>([&](auto N2_) { b[decltype(N2_)::value] = t[decltype(N2_)::value * A + k1]; });
                Dft<B, DIR, C>::run(b);
                sfor<0, B>([&](auto K2_) { v[k1 + A * decltype(K2_)::value] = b[decltype(K2_)::value]; });
            });
        }
    }
};

// ---------------------------------------------------------------------------
// Radix sequences
// ---------------------------------------------------------------------------
template <int... Rs> struct Seq {};

template <class In, class Out> struct RevImpl;
template <int... Out> struct RevImpl<Seq<>, Seq<Out...>> { using type = Seq<Out...>; };
template <int H, int... T, int... Out> struct RevImpl<Seq<H, T...>, Seq<Out...>> {
    using type = typename RevImpl<Seq<T...>, Seq<H, Out...>>::type;
};
template <class S> using Reverse = typename RevImpl<S, Seq<>>::type;

template <class S> struct SeqInfo;
template <int H, int... T> struct SeqInfo<Seq<H, T...>> {
    static constexpr int first = H;
    static constexpr int last = sizeof...(T) == 0 ? H : SeqInfo<Seq<T...>>::last;
    static constexpr int min_r = (sizeof...(T) == 0 || H < SeqInfo<Seq<T...>>::min_r) ? H : SeqInfo<Seq<T...>>::min_r;
    static constexpr int max_r = (sizeof...(T) == 0 || H > SeqInfo<Seq<T...>>::max_r) ? H : SeqInfo<Seq<T...>>::max_r;
    static constexpr int product = H * SeqInfo<Seq<T...>>::product;
    static constexpr int stages = 1 + sizeof...(T);
};
template <> struct SeqInfo<Seq<>> {
    static constexpr int first = 1, last = 1, min_r = 1 << 30, max_r = 0, product = 1, stages = 0;
};

// ---------------------------------------------------------------------------
// Shared-memory exchange layout.  Complex values are stored interleaved
// (one 64-bit access per element).  The exchange after a stage with group
// size P = Ns * R inserts q padding elements after every group of P:
//   padded(i) = i + q * (i / P).
// The next stage reads x[j + m NB'] with NB' = N / R' a multiple of P, so
// both sides stay "per-thread base + compile-time offset".  q is chosen so
// that the 16 threads of each 64-bit access phase hit distinct bank pairs:
// an odd element stride when Ns = 1, and consecutive banks across groups
// (Ns R + q = Ns mod 16) otherwise.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pad_q(int Ns, int R)
{
    return Ns == 1 ? ((R % 2 == 0) ? 1 : 0) : (((Ns * (1 - R)) % 16) + 16) % 16;
}

// elements of shared memory one chain's exchanges touch
template <int... Rs>
__host__ __device__ constexpr int chain_extent()
{
    constexpr int S = sizeof...(Rs);
    const int r[S] = {Rs...};
    int n = 1;
    for (int s = 0; s < S; ++s) n *= r[s];
    int ext = n, Ns = 1;
    for (int s = 0; s + 1 < S; ++s) {
        const int P = Ns * r[s], q = pad_q(Ns, r[s]);
        const int e = (n - 1) + q * ((n - 1) / P) + 1;
        ext = e > ext ? e : ext;
        Ns = P;
    }
    return ext;
}
template <class S> struct ChainExtent;
template <int... Rs> struct ChainExtent<Seq<Rs...>> {
    static constexpr int value = chain_extent<Rs...>();
};

// ---------------------------------------------------------------------------
// Stage chain in FP32.  TT threads cooperate on one transform; in a stage
// with NB = N/R butterflies, thread t owns butterflies j = t + e TT for
// e < E = ceil(NB / TT) (j < NB).  `run` takes the inputs of the first
// stage in v[e] (thread t holds x[j + m N/R]), runs every stage, exchanging
// through shared memory `sm` between stages, and hands the last stage's
// outputs (v[e] holds y[j + m N/R_last]) to `fin(v, t)`.
// Every thread of the block must call it (it contains barriers).
// ---------------------------------------------------------------------------
// Double buffering (DB): exchange number x of the block's sequence uses
// buffer (BUF + x) mod 2 (sm and sm + bstride).  Consecutive exchanges then
// use different buffers, so the write of an exchange only has to wait for
// the readers of the exchange two before it -- which finished before the
// previous exchange's barrier -- and one barrier per exchange suffices.
template <int N, int DIR, int Ns, int SIdx, int TT, class S, bool DB = false, int BUF = 0> struct Chain;

template <int N, int DIR, int Ns, int SIdx, int TT, int R, int... Rest, bool DB, int BUF>
struct Chain<N, DIR, Ns, SIdx, TT, Seq<R, Rest...>, DB, BUF> {
    static constexpr int NB = N / R;
    static constexpr int E = (NB + TT - 1) / TT;
    static constexpr int EXCHANGES = sizeof...(Rest);

    template <class Fin>
    __device__ __forceinline__ static void run(float2 (&v)[E][R], int t, float2* sm,
                                               const TwChain& tw, Fin&& fin, int bstride = 0)
    {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int j = t + e * TT;
            if (j < NB) {
                if constexpr (Ns > 1) {
                    const float2* tab = tw.p[SIdx];
                    // opaque to the optimiser: keeps the table loads inside
                    // loops that repeat a chain instead of hoisting every
                    // stage's twiddles into registers across iterations
                    asm volatile("" : "+l"(tab));
                    tab += j % Ns;
#pragma unroll
                    for (int m = 1; m < R; ++m) {
                        float2 w = __ldg(tab + (m - 1) * Ns);
                        if constexpr (DIR > 0) w.y = -w.y;
                        v[e][m] = cmul(v[e][m], w);
                    }
                }
                Dft<R, DIR, float2>::run(v[e]);
            }
        }
        if constexpr (sizeof...(Rest) == 0) {
            fin(v, t);
        } else {
            using Next = Chain<N, DIR, Ns * R, SIdx + 1, TT, Seq<Rest...>, DB, BUF>;
            float2* xb = (DB && ((BUF + SIdx) & 1)) ? sm + bstride : sm;
            constexpr int R2 = SeqInfo<Seq<Rest...>>::first;
            constexpr int NB2 = N / R2;
            constexpr int P = Ns * R;
            constexpr int q = pad_q(Ns, R);
            static_assert(NB2 % P == 0, "reader stride must be a multiple of the group size");
            constexpr int rstride = NB2 + q * (NB2 / P);
            if constexpr (!DB) __syncthreads();  // earlier readers of sm are done
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int j = t + e * TT;
                if (j < NB) {
                    float2* w0 = xb + (j / Ns) * (P + q) + (j % Ns);
#pragma unroll
                    for (int m = 0; m < R; ++m) w0[m * Ns] = v[e][m];
                }
            }
            __syncthreads();
            float2 w[Next::E][R2];
#pragma unroll
            for (int e = 0; e < Next::E; ++e) {
                const int j = t + e * TT;
                if (j < NB2) {
                    const float2* r0 = xb + j + q * (j / P);
#pragma unroll
                    for (int m = 0; m < R2; ++m) w[e][m] = r0[m * rstride];
                }
            }
            Next::run(w, t, sm, tw, fin, bstride);
        }
    }
};

}  // namespace lpk
