// The three FP32 passes of the Fourier-domain convolution (Sec. 2.3 Eq. (9),
// workflow of Sec. 2.5 / Fig. 1) on the in-place engine of fft2.cuh: zero
// padding is implicit, the spectrum product sits between the forward and the
// inverse column transform, and the crop is a predicate on the last stores.
//
//   P1  rows:     two real rows a, b packed as z = a + i b, forward FFT of
//                 length Nx, split into the half spectra of a and b
//                 (Hermitian symmetry), stored for columns c <= Nx/2.
//   P2  columns:  per column, forward FFT of length Ny of the h stored rows
//                 (rows >= h are the zero padding), product with the PSF
//                 spectrum K^ (pre-scaled by 1/(2 Ny Nx)), inverse FFT, store
//                 the rows of the crop window.
//   P3  rows:     Hermitian extension of two rows' half spectra packed as
//                 Z = A + i B, inverse FFT, real part -> row a, imaginary part
//                 -> row b, store the crop columns.
//
// Work units.  The two-transform form (CP) of a pass takes two units per
// thread block: two columns (P2) or two row pairs (P1, P3); the
// single-transform form (float2) takes one.  A block of T threads holds one
// transform buffer of N elements in shared memory.
//
// Layout of the intermediate half spectra (T: written by P1, read by P2;
// U: written by P2, read by P3), "column pairs": columns c = 2 q and 2 q + 1
// form pair q, and element (pair q, row r) is one float4
//   {re X_r[2q], re X_r[2q+1], im X_r[2q], im X_r[2q+1]}
// at index q * ld + r (ld = rows stored per pair, a multiple of 4).  A pair's
// rows are contiguous, so the column pass reads and writes each of its two
// columns' data as one contiguous run, and the row passes move 16 bytes per
// column pair and row (64 contiguous bytes for the four rows of a
// two-transform block).  The column past the last one (odd Nx/2 + 1) is
// written by P1 and never read.
//
// FP32 PSF spectra are stored for the column pass: per column pair q, Ny
// entries (leading dimension ldK) in the position order of the column
// transform (entry p holds the frequency the forward transform leaves at
// position p), each {K[2q], K[2q+1]} (real spectrum) or {re K[2q], re K[2q+1],
// im K[2q], im K[2q+1]} (complex spectrum).  The product then reads the
// spectrum in the order the transform holds its values: contiguous per
// butterfly, coalesced across the threads.
#pragma once

#include "conv_kernels.cuh"
#include "fft2.cuh"

namespace lpk {

// rows stored per column pair: a multiple of 4 (the four rows of a
// two-transform row-pass block)
__host__ __device__ constexpr long long pair_ld(long long rows) { return (rows + 3) / 4 * 4; }
__host__ __device__ constexpr long long pair_count(long long ncols) { return (ncols + 1) / 2; }

struct P1v2Args {
    const float* L;
    long long ldl;
    int H, W;
    float4* T;
    long long ldT;
    int unit0, units;  // units [unit0, units): row quads (CP) or row pairs (float2)
    int ncols;         // Nx/2 + 1
    TwTab2 tw;         // row-length tables
};

struct P2v2Args {
    const float4* T;
    long long ldT;
    int H;
    const void* K[kMaxSpectraPerLaunch];
    long long ldK;
    int nspec;
    float4* U;
    long long ldU;
    long long specU;  // float4 elements between consecutive spectra's U
    int r0;           // first kept row (mod Ny) of the inverse output
    int Hout;         // kept rows
    int ncols;
    float4* park;     // batched form: forward spectra, N float4 per block
    TwTab2 tw;        // column-length tables
};

struct P3v2Args {
    const float4* U;
    long long ldU;
    long long specU;
    int Hout;
    int unit0, units;  // output row quads (CP) or row pairs (float2)
    float* out[kMaxSpectraPerLaunch];
    long long ldo;
    int c0;  // first kept column (mod Nx)
    int Wout;
    int ncols;
    TwTab2 tw;
};

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// ---------------------------------------------------------------------------
// element access of the column-pair layout
// ---------------------------------------------------------------------------
__device__ __forceinline__ CP cp_of(float4 q) { return CP{make_float2(q.x, q.y), make_float2(q.z, q.w)}; }
__device__ __forceinline__ float4 f4_of(const CP& v) { return make_float4(v.x.x, v.x.y, v.y.x, v.y.y); }

// ---------------------------------------------------------------------------
// P1: forward row transform
// ---------------------------------------------------------------------------
// Split of the packed spectrum Z (positions of the forward transform) into
// the half spectra of the packed rows: 2 X_a[c] = Z[c] + conj Z[N-c],
// 2 X_b[c] = -i (Z[c] - conj Z[N-c]).
template <class C>
__device__ __forceinline__ void unpack_pair(const C& zc, const C& zm, C& xa, C& xb);
template <>
__device__ __forceinline__ void unpack_pair<CP>(const CP& zc, const CP& zm, CP& xa, CP& xb)
{
    xa = CP{add2(zc.x, zm.x), sub2(zc.y, zm.y)};
    xb = CP{add2(zc.y, zm.y), sub2(zm.x, zc.x)};
}
template <>
__device__ __forceinline__ void unpack_pair<float2>(const float2& zc, const float2& zm, float2& xa, float2& xb)
{
    xa = make_float2(zc.x + zm.x, zc.y - zm.y);
    xb = make_float2(zc.y + zm.y, zm.x - zc.x);
}

template <class G, int T, int MINB, class C>
__global__ void __launch_bounds__(T, MINB) p1v2(const P1v2Args a)
{
    pdl_begin();
    constexpr int N = G::B(0);
    constexpr bool PAIR = std::is_same<C, CP>::value;
    constexpr int ROWS = PAIR ? 4 : 2;  // map rows per block
    extern __shared__ float4 smem_v2[];
    C* X = reinterpret_cast<C*>(smem_v2);
    float* Xf = reinterpret_cast<float*>(smem_v2);
    const int t = threadIdx.x;
    const int unit = a.unit0 + blockIdx.x;
    const int r0 = ROWS * unit;
    // element n of the packed transforms: rows (a_A, a_B, b_A, b_B) of column
    // n for two transforms, (a, b) for one; columns >= W and rows >= H are 0
    constexpr int SLOT[4] = {0, 2, 1, 3};  // map row i -> float of the element
    for (int n = t; n < N; n += T) {
#pragma unroll
        for (int i = 0; i < ROWS; ++i) {
            float* dst = Xf + (size_t)n * ROWS + (PAIR ? SLOT[i] : i);
            if (n < a.W && r0 + i < a.H) cpa4(dst, a.L + (long long)(r0 + i) * a.ldl + n);
            else *dst = 0.f;
        }
    }
    cpa_wait_all();
    __syncthreads();
    ip_forward<G, 0, G::S, T, C>(X, t, a.tw);
    // half spectra of the block's rows, by column pair
    const int ncp = (int)pair_count(a.ncols);
#pragma unroll 2
    for (int q = t; q < ncp; q += T) {
        C xa[2], xb[2];
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int c = 2 * q + l;
            const int cm = (c == 0) ? 0 : N - c;
            const C zc = X[__ldg(a.tw.pos + (c < N ? c : 0))];
            const C zm = X[__ldg(a.tw.pos + cm)];
            unpack_pair<C>(zc, zm, xa[l], xb[l]);
        }
        float4* dst = a.T + (long long)q * a.ldT + r0;
        if constexpr (PAIR) {
            // rows r0 .. r0+3: a_A, b_A, a_B, b_B (lane 0 / 1 of the pairs)
            dst[0] = make_float4(xa[0].x.x, xa[1].x.x, xa[0].y.x, xa[1].y.x);
            dst[1] = make_float4(xb[0].x.x, xb[1].x.x, xb[0].y.x, xb[1].y.x);
            dst[2] = make_float4(xa[0].x.y, xa[1].x.y, xa[0].y.y, xa[1].y.y);
            dst[3] = make_float4(xb[0].x.y, xb[1].x.y, xb[0].y.y, xb[1].y.y);
        } else {
            dst[0] = make_float4(xa[0].x, xa[1].x, xa[0].y, xa[1].y);
            dst[1] = make_float4(xb[0].x, xb[1].x, xb[0].y, xb[1].y);
        }
    }
}

// ---------------------------------------------------------------------------
// P2: column transform with the spectrum product
// ---------------------------------------------------------------------------
// The unit's spectrum in the column-pass layout (position order): the pair
// q's entries (two transforms) or column c's lane of them (one transform).
template <class C, bool KREAL>
struct SpecIo;
template <bool KREAL>
struct SpecIo<CP, KREAL> {
    const char* base;
    __device__ __forceinline__ SpecIo(const void* K, long long ldK, int unit)
        : base(static_cast<const char*>(K) + (size_t)unit * ldK * (KREAL ? 8 : 16)) {}
    __device__ __forceinline__ void apply(CP& v, int p) const
    {
        if constexpr (KREAL) {
            const float2 kk = __ldg(reinterpret_cast<const float2*>(base) + p);
            v.x = mul2(v.x, kk);
            v.y = mul2(v.y, kk);
        } else {
            const float4 k4 = __ldg(reinterpret_cast<const float4*>(base) + p);
            const float2 kr = make_float2(k4.x, k4.y), ki = make_float2(k4.z, k4.w);
            const CP r{fma2(v.y, neg2(ki), mul2(v.x, kr)), fma2(v.x, ki, mul2(v.y, kr))};
            v = r;
        }
    }
};
template <bool KREAL>
struct SpecIo<float2, KREAL> {
    const float* base;
    __device__ __forceinline__ SpecIo(const void* K, long long ldK, int c)
        : base(static_cast<const float*>(K) + (size_t)(c >> 1) * ldK * (KREAL ? 2 : 4) + (c & 1)) {}
    __device__ __forceinline__ void apply(float2& v, int p) const
    {
        if constexpr (KREAL) {
            const float k = __ldg(base + 2 * p);
            v = make_float2(v.x * k, v.y * k);
        } else {
            const float kr = __ldg(base + 4 * p), ki = __ldg(base + 4 * p + 2);
            v = make_float2(v.x * kr - v.y * ki, v.x * ki + v.y * kr);
        }
    }
};

// The unit's column data: pair q (CP) or column c (float2: lane c & 1).
template <class C>
struct ColIo;
template <>
struct ColIo<CP> {
    const float4* src;
    float4* dst;
    __device__ __forceinline__ ColIo(const float4* T, long long ldT, float4* U, long long ldU, int unit)
        : src(T + (long long)unit * ldT), dst(U + (long long)unit * ldU) {}
    __device__ __forceinline__ void stage(CP* X, int r) const { cpa16(X + r, src + r); }
    __device__ __forceinline__ void store(int r, const CP& v) const { dst[r] = f4_of(v); }
};
template <>
struct ColIo<float2> {
    const float* src;
    float* dst;
    __device__ __forceinline__ ColIo(const float4* T, long long ldT, float4* U, long long ldU, int c)
        : src(reinterpret_cast<const float*>(T + (long long)(c >> 1) * ldT) + (c & 1)),
          dst(reinterpret_cast<float*>(U + (long long)(c >> 1) * ldU) + (c & 1)) {}
    __device__ __forceinline__ void stage(float2* X, int r) const
    {
        cpa4(reinterpret_cast<float*>(X + r), src + 4 * r);
        cpa4(reinterpret_cast<float*>(X + r) + 1, src + 4 * r + 2);
    }
    __device__ __forceinline__ void store(int r, const float2& v) const
    {
        dst[4 * r] = v.x;
        dst[4 * r + 2] = v.y;
    }
};

template <class C>
__device__ __forceinline__ C czero()
{
    if constexpr (std::is_same<C, CP>::value) return CP{make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    else return make_float2(0.f, 0.f);
}

// the column (pair) rows [0, H) staged into X, zeros up to N
template <int N, int T, class C>
__device__ __forceinline__ void stage_column(C* X, const ColIo<C>& io, int H, int t)
{
    for (int r = t; r < N; r += T) {
        if (r < H) io.stage(X, r);
        else X[r] = czero<C>();
    }
    cpa_wait_all();
    __syncthreads();
}

template <class G, int T, int MINB, class C, bool KREAL>
__global__ void __launch_bounds__(T, MINB) p2v2(const __grid_constant__ P2v2Args a)
{
    pdl_begin();
    constexpr int N = G::B(0);
    extern __shared__ float4 smem_v2[];
    C* X = reinterpret_cast<C*>(smem_v2);
    const int t = threadIdx.x;
    const int unit = blockIdx.x;
    const ColIo<C> io(a.T, a.ldT, a.U, a.ldU, unit);
    stage_column<N, T, C>(X, io, a.H, t);
    ip_forward<G, 0, G::S - 1, T, C>(X, t, a.tw);
    const SpecIo<C, KREAL> sp(a.K[0], a.ldK, unit);
    ip_middle<G, T, C>(X, t, [&](int p, C& v) { sp.apply(v, p); });
    __syncthreads();
    ip_inverse<G, 1, G::S - 1, T, C>(X, t, a.tw);
    ip_last_inverse<G, T, C>(X, t, a.tw, [&](int n, const C& v) {
        int rr = n - a.r0;
        if (rr < 0) rr += N;
        if (rr < a.Hout) io.store(rr, v);
    });
}

// Several spectra from one forward column transform: the forward spectrum
// is parked in global memory (a.park, N elements per block, L2-resident
// while the block runs) and every spectrum's product and inverse start from
// it.
template <class G, int T, int MINB, class C, bool KREAL>
__global__ void __launch_bounds__(T, MINB) p2v2_multi(const __grid_constant__ P2v2Args a)
{
    pdl_begin();
    constexpr int N = G::B(0);
    constexpr int R = G::RL, NB = N / R;
    constexpr int E = (NB + T - 1) / T;
    extern __shared__ float4 smem_v2[];
    C* X = reinterpret_cast<C*>(smem_v2);
    C* park = reinterpret_cast<C*>(a.park) + (size_t)blockIdx.x * N;
    const int t = threadIdx.x;
    const int unit = blockIdx.x;
    const ColIo<C> io(a.T, a.ldT, a.U, a.ldU, unit);
    stage_column<N, T, C>(X, io, a.H, t);
    ip_forward<G, 0, G::S - 1, T, C>(X, t, a.tw);
    // the forward's last stage, parked (each thread later reads back only
    // the elements it wrote, so no barrier is needed around the park)
#pragma unroll 1
    for (int e = 0; e < E; ++e) {
        const int blk = t + e * T;
        if (NB % T != 0 && blk >= NB) break;
        C v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = X[blk * R + k];
        D2<R, -1, C>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) park[blk * R + k] = v[k];
    }
    for (int s = 0; s < a.nspec; ++s) {
        const SpecIo<C, KREAL> sp(a.K[s], a.ldK, unit);
        __syncthreads();  // the previous spectrum's last stage has read X
#pragma unroll 1
        for (int e = 0; e < E; ++e) {
            const int blk = t + e * T;
            if (NB % T != 0 && blk >= NB) break;
            C v[R];
#pragma unroll
            for (int k = 0; k < R; ++k) v[k] = park[blk * R + k];
#pragma unroll
            for (int k = 0; k < R; ++k) sp.apply(v[k], blk * R + k);
            D2<R, +1, C>::run(v);
#pragma unroll
            for (int k = 0; k < R; ++k) X[blk * R + k] = v[k];
        }
        __syncthreads();
        ip_inverse<G, 1, G::S - 1, T, C>(X, t, a.tw);
        const ColIo<C> os(a.T, a.ldT, a.U + (long long)s * a.specU, a.ldU, unit);
        ip_last_inverse<G, T, C>(X, t, a.tw, [&](int n, const C& v) {
            int rr = n - a.r0;
            if (rr < 0) rr += N;
            if (rr < a.Hout) os.store(rr, v);
        });
    }
}

// Sec. 2.2 Eq. (4): several source classes, one PSF each.  Each class's
// column is transformed forward and multiplied by its spectrum; the products
// are summed (in a.park, N elements per block) before one inverse transform.
struct P2Mv2Args {
    P2v2Args a;           // a.K[t]: spectrum of class t; a.T unused
    const float4* T[kMaxSpectraPerLaunch];  // class maps' half spectra
    int nclass;
};

template <class G, int T, int MINB, class C, bool KREAL>
__global__ void __launch_bounds__(T, MINB) p2v2_multiclass(const __grid_constant__ P2Mv2Args m)
{
    pdl_begin();
    const P2v2Args& a = m.a;
    constexpr int N = G::B(0);
    constexpr int R = G::RL, NB = N / R;
    constexpr int E = (NB + T - 1) / T;
    extern __shared__ float4 smem_v2[];
    C* X = reinterpret_cast<C*>(smem_v2);
    C* acc = reinterpret_cast<C*>(a.park) + (size_t)blockIdx.x * N;
    const int t = threadIdx.x;
    const int unit = blockIdx.x;
    for (int q = 0; q < m.nclass; ++q) {
        const ColIo<C> io(m.T[q], a.ldT, a.U, a.ldU, unit);
        if (q > 0) __syncthreads();  // the previous class's last stage has read X
        stage_column<N, T, C>(X, io, a.H, t);
        ip_forward<G, 0, G::S - 1, T, C>(X, t, a.tw);
        const SpecIo<C, KREAL> sp(a.K[q], a.ldK, unit);
        // each thread accumulates only the elements it owns
#pragma unroll 1
        for (int e = 0; e < E; ++e) {
            const int blk = t + e * T;
            if (NB % T != 0 && blk >= NB) break;
            C v[R];
#pragma unroll
            for (int k = 0; k < R; ++k) v[k] = X[blk * R + k];
            D2<R, -1, C>::run(v);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                sp.apply(v[k], blk * R + k);
                acc[blk * R + k] = q == 0 ? v[k] : c_add(acc[blk * R + k], v[k]);
            }
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int e = 0; e < E; ++e) {
        const int blk = t + e * T;
        if (NB % T != 0 && blk >= NB) break;
        C v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = acc[blk * R + k];
        D2<R, +1, C>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) X[blk * R + k] = v[k];
    }
    __syncthreads();
    ip_inverse<G, 1, G::S - 1, T, C>(X, t, a.tw);
    const ColIo<C> os(m.T[0], a.ldT, a.U, a.ldU, unit);
    ip_last_inverse<G, T, C>(X, t, a.tw, [&](int n, const C& v) {
        int rr = n - a.r0;
        if (rr < 0) rr += N;
        if (rr < a.Hout) os.store(rr, v);
    });
}

// ---------------------------------------------------------------------------
// P3: inverse row transform and crop
// ---------------------------------------------------------------------------
// Packed inverse inputs of frequency c <= N/2 and N - c from the half
// spectra A, B of the two rows: Z[c] = A + i B, Z[N-c] = conj A + i conj B.
__device__ __forceinline__ void pack_pair(float2 A, float2 B, float2& zc, float2& zm)
{
    zc = make_float2(A.x - B.y, A.y + B.x);
    zm = make_float2(A.x + B.y, B.x - A.y);
}

template <class G, int T, int MINB, class C>
__global__ void __launch_bounds__(T, MINB) p3v2(const P3v2Args a)
{
    pdl_begin();
    constexpr int N = G::B(0);
    constexpr bool PAIR = std::is_same<C, CP>::value;
    constexpr int ROWS = PAIR ? 4 : 2;
    extern __shared__ float4 smem_v2[];
    C* X = reinterpret_cast<C*>(smem_v2);
    const int t = threadIdx.x;
    const int unit = a.unit0 + blockIdx.x;
    const int sidx = blockIdx.y;
    const int r0 = ROWS * unit;
    const float4* Us = a.U + (long long)sidx * a.specU;
    const int ncp = (int)pair_count(a.ncols);
#pragma unroll 2
    for (int q = t; q < ncp; q += T) {
        float4 u[ROWS];
#pragma unroll
        for (int i = 0; i < ROWS; ++i)
            u[i] = (r0 + i < a.Hout) ? ldg4(Us + (long long)q * a.ldU + r0 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            const int c = 2 * q + l;
            if (c >= a.ncols) break;
            float2 zc[ROWS / 2], zm[ROWS / 2];
#pragma unroll
            for (int p = 0; p < ROWS / 2; ++p) {
                const float4 A4 = u[2 * p], B4 = u[2 * p + 1];
                const float2 A = l ? make_float2(A4.y, A4.w) : make_float2(A4.x, A4.z);
                const float2 B = l ? make_float2(B4.y, B4.w) : make_float2(B4.x, B4.z);
                pack_pair(A, B, zc[p], zm[p]);
            }
            C vc, vm;
            if constexpr (PAIR) {
                vc = CP{make_float2(zc[0].x, zc[1].x), make_float2(zc[0].y, zc[1].y)};
                vm = CP{make_float2(zm[0].x, zm[1].x), make_float2(zm[0].y, zm[1].y)};
            } else {
                vc = zc[0];
                vm = zm[0];
            }
            X[__ldg(a.tw.pos + c)] = vc;
            if (c != 0 && 2 * c != N) X[__ldg(a.tw.pos + (N - c))] = vm;
        }
    }
    __syncthreads();
    ip_inverse<G, 1, G::S, T, C>(X, t, a.tw);
    float* o[ROWS];
    bool ok[ROWS];
#pragma unroll
    for (int i = 0; i < ROWS; ++i) {
        ok[i] = r0 + i < a.Hout;
        o[i] = a.out[sidx] + (long long)(ok[i] ? r0 + i : 0) * a.ldo;
    }
    ip_last_inverse<G, T, C>(X, t, a.tw, [&](int n, const C& v) {
        int cc = n - a.c0;
        if (cc < 0) cc += N;
        if (cc >= a.Wout) return;
        if constexpr (PAIR) {
            if (ok[0]) o[0][cc] = v.x.x;
            if (ok[1]) o[1][cc] = v.y.x;
            if (ok[2]) o[2][cc] = v.x.y;
            if (ok[3]) o[3][cc] = v.y.y;
        } else {
            if (ok[0]) o[0][cc] = v.x;
            if (ok[1]) o[1][cc] = v.y;
        }
    });
}

}  // namespace lpk
