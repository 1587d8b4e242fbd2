// The three FP32 passes of the Fourier-domain convolution (Sec. 2.3 Eq. (9),
// workflow of Sec. 2.5 / Fig. 1): zero padding is implicit, the spectrum
// product sits between the forward and inverse column transforms, and the
// crop is a predicate on the last stores.
//
//   P1  rows:    two real rows a, b packed as z = a + i b, length-Nx forward
//                FFT, split into the half spectra of a and b (Hermitian
//                symmetry), stored by column c in [0, Nx/2] (column-blocked
//                layout, below).
//   P2  columns: per column c, length-Ny forward FFT of T[c][0..H) (rows
//                >= H are the zero padding), multiply by the PSF spectrum
//                K^[c][.] (pre-scaled by 1/(2 Ny Nx)), inverse FFT, keep the
//                output rows of the crop window.  With n spectra the batched
//                kernel parks the forward result in shared memory and reuses
//                it n times; plans may instead run one pass per spectrum.
//   P3  rows:    Hermitian extension of two rows' half spectra packed as
//                Z = A + i B, length-Nx inverse FFT, real part -> row a,
//                imaginary part -> row b, keep the crop columns.
//
// Layouts (element = complex64 unless stated):
//   L    FP32, row-major H x W, leading dimension ldl (elements)
//   T    the row pass's half spectra, column-blocked (below): ldT >= 2 ceil(H/2)
//        elements per column, Nx/2+1 columns rounded up to a multiple of kTCB
//   K^   (Nx/2+1) rows of ldK elements: FP32 (point-symmetric PSF, real
//        spectrum) or complex64
//   U    per spectrum, column-blocked (below): ldU >= 2 ceil(Hout/2) elements per
//        column, Nx/2+1 columns rounded up to a multiple of kUCB
//   out  FP32 row-major Hout x Wout, leading dimension ldo
#pragma once

#include "fft_core.cuh"

namespace lpk {

// Column-blocked layout of the intermediate half spectra T and U.  Element
// (column c, row pair p) is a float4 {row 2p, row 2p+1} of column c; the
// columns are grouped in blocks of CB, and within a block the CB columns'
// float4 of one row pair sit side by side:
//   float4 index ((c / CB) * ldq + p) * CB + c mod CB,  ldq = ld / 2,
// with ld the (even) number of rows stored per column.  The row passes,
// which handle all columns of one row pair, then move 16 CB contiguous
// bytes per column block instead of 16 scattered ones; the column pass
// reads / writes a column at a 16 CB-byte stride.  Measured at 4704^2 for
// T: row pass 74 -> 58 us, column pass 68 -> 70 us with CB = 2 (with 4 / 8:
// 55.5 / 53.7 and 74 / 80 us).  The CB-1 columns past the last one that
// padding adds to a partial last block are allocated and never touched.
template <int CB>
__host__ __device__ constexpr long long blk_cols_alloc(long long ncols) { return (ncols + CB - 1) / CB * CB; }
template <int CB>
__host__ __device__ __forceinline__ long long blk_index4(int c, long long p, long long ldq)
{
    return ((long long)(c / CB) * ldq + p) * CB + (c % CB);
}
// row r of a column, in float2 from the column's row 0
template <int CB>
__host__ __device__ __forceinline__ long long blk_row(int r) { return (long long)(r >> 1) * (2 * CB) + (r & 1); }

constexpr int kTCB = 2;  // T: written by the forward row pass, read by the column pass
// U: written by the column pass, read by the inverse row pass.  Measured
// (column / inverse row pass, us), blocks of 1 / 2 / 4:
//   4704^2:   70.3 / 72.4 / 75.5  and  59.7 / 57.0 / 54.9
//   17280^2:  1049 / 1142 / 1145  and  1225 / 994 / 851
constexpr int kUCB = 4;
__host__ __device__ constexpr long long t_cols_alloc(long long ncols) { return blk_cols_alloc<kTCB>(ncols); }
__host__ __device__ constexpr long long u_cols_alloc(long long ncols) { return blk_cols_alloc<kUCB>(ncols); }
__host__ __device__ __forceinline__ long long t_index4(int c, long long p, long long ldq) { return blk_index4<kTCB>(c, p, ldq); }
__host__ __device__ __forceinline__ long long u_index4(int c, long long p, long long ldq) { return blk_index4<kUCB>(c, p, ldq); }
__host__ __device__ __forceinline__ long long t_row(int r) { return blk_row<kTCB>(r); }
// offset of row j + m S from row j's when S is even (the pair index moves by
// m S / 2, the row parity stays): a compile-time multiple of m
template <int S>
__host__ __device__ constexpr long long t_row_step() { return (long long)(S / 2) * 2 * kTCB; }
__host__ __device__ __forceinline__ long long u_row(int r) { return blk_row<kUCB>(r); }
// float2 pointer to row 0 of column c
__host__ __device__ __forceinline__ const float2* t_column(const float2* T, long long ldT, int c)
{
    return T + 2 * t_index4(c, 0, ldT / 2);
}
__host__ __device__ __forceinline__ float2* u_column(float2* U, long long ldU, int c)
{
    return U + 2 * u_index4(c, 0, ldU / 2);
}

constexpr int kMaxSpectraPerLaunch = 32;

struct P1Args {
    const float* L;
    long long ldl;
    int H, W;
    int Wst;    // staged row length (floats): W rounded up to a multiple of 4
    int vec16;  // rows can be copied in 16-byte pieces (aligned base, ldl % 4 == 0, W % 4 == 0)
    float2* T;
    long long ldT;
    int pair0;   // first row pair of this launch (pairs pair0 .. npairs-1)
    int npairs;  // ceil(H/2)
    int ncols;   // Nx/2 + 1
    TwChain tw;  // forward chain of the row plan
    int* err;            // device status word (debug builds: bounds checks)
    long long t_elems;   // float2 elements of the T buffer
};

struct P2Args {
    const float2* T;
    long long ldT;
    int H;
    const void* K[kMaxSpectraPerLaunch];
    long long ldK;
    int nspec;
    float2* U;
    long long ldU;
    long long specU;  // elements between consecutive spectra's U blocks
    int r0;           // first kept row (mod Ny) of the inverse output
    int Hout;         // kept rows
    int HoutPad;      // 2 ceil(Hout/2): rows written (the extra one is zero)
    int ncols;
    TwChain twf, twi;  // forward and reversed chains of the column plan
    float2* park;      // batched pass: forward column spectra, N per column
    int ahead;         // column distance of the T prefetch into L2 (0: none)
    int* err;              // device status word (debug builds: bounds checks)
    long long t_elems;     // float2 elements of the T buffer
    long long u_elems;     // float2 elements of U from a.U on (all spectra of the launch)
    long long k_elems;     // spectrum values (floats or float2) of each spectrum
    long long park_elems;  // float2 elements of the park area (0 without one)
};

struct P3Args {
    const float2* U;
    long long ldU;
    long long specU;
    int Hout, npairs;
    int pair0;  // first output row pair of this launch
    float* out[kMaxSpectraPerLaunch];
    long long ldo;
    int c0;  // first kept column (mod Nx)
    int Wout;
    int ncols;
    TwChain tw;  // reversed chain of the row plan
    int* err;           // device status word (debug builds: bounds checks)
    long long u_elems;  // float2 elements of U from a.U on (all spectra of the launch)
};

// Debug builds (LP_DEBUG=1, a library of their own): before a work unit
// touches global memory, its block checks the unit's whole extent in every
// buffer against the sizes the host passed; a unit outside them sets bit 3
// of the device status word and is skipped (no assert or trap, so the
// context stays usable).  Release builds compile the checks away.
#ifndef LP_DEBUG
#define LP_DEBUG 0
#endif
constexpr int kDevErrBounds = 8;

__device__ __forceinline__ bool lp_checked(int* err, bool ok)
{
#if LP_DEBUG
    if (!ok && threadIdx.x == 0) atomicOr(err, kDevErrBounds);
    return ok;
#else
    (void)err;
    (void)ok;
    return true;
#endif
}

// P1 unit: rows 2 pair, 2 pair + 1 of L, and row pair `pair` of every column of T
__device__ __forceinline__ bool p1_unit_ok(const P1Args& a, int pair)
{
#if LP_DEBUG
    const long long ldq = a.ldT / 2;
    return lp_checked(a.err, pair >= 0 && 2 * pair < a.H && pair < ldq && a.W <= a.ldl &&
                                 2 * (t_index4(a.ncols - 1, pair, ldq) + 1) <= a.t_elems);
#else
    (void)a;
    (void)pair;
    return true;
#endif
}

// P2 unit: column c of T (all ldT rows), of each spectrum, of each of the
// launch's U blocks (HoutPad rows) and of the park area
__device__ __forceinline__ bool p2_column_ok(const P2Args& a, int c, int n, int kw)
{
#if LP_DEBUG
    const bool t_ok = 2 * t_index4(c, 0, a.ldT / 2) + t_row((int)a.ldT - 1) < a.t_elems && a.H <= a.ldT;
    const bool k_ok = (long long)(c + 1) * a.ldK <= a.k_elems && n <= a.ldK;
    const bool u_ok = a.HoutPad <= a.ldU &&
                      (long long)(a.nspec - 1) * a.specU + 2 * u_index4(c, 0, a.ldU / 2) + u_row(a.HoutPad - 1) <
                          a.u_elems;
    const bool p_ok = a.park == nullptr || (long long)(c + 1) * n <= a.park_elems;
    (void)kw;
    return lp_checked(a.err, c >= 0 && c < a.ncols && t_ok && k_ok && u_ok && p_ok);
#else
    (void)a;
    (void)c;
    (void)n;
    (void)kw;
    return true;
#endif
}

// P3 unit: row pair `pair` of every column of U block sidx, rows 2 pair,
// 2 pair + 1 of out[sidx]
__device__ __forceinline__ bool p3_unit_ok(const P3Args& a, int pair, int sidx)
{
#if LP_DEBUG
    const long long ldq = a.ldU / 2;
    return lp_checked(a.err, pair >= 0 && 2 * pair < a.Hout && pair < ldq && a.out[sidx] != nullptr &&
                                 a.Wout <= a.ldo &&
                                 (long long)sidx * a.specU + 2 * (u_index4(a.ncols - 1, pair, ldq) + 1) <=
                                     a.u_elems);
#else
    (void)a;
    (void)pair;
    (void)sidx;
    return true;
#endif
}

template <int N, class FwdSeq, int TT_ = 0>
struct Plan {
    using Fwd = FwdSeq;
    using Inv = Reverse<FwdSeq>;
    static_assert(SeqInfo<Fwd>::product == N, "radices must multiply to N");
    static constexpr int R0 = SeqInfo<Fwd>::first;   // first forward radix
    static constexpr int RL = SeqInfo<Fwd>::last;    // last forward radix
    // threads per transform: one butterfly per thread in every stage by
    // default (N / smallest radix, rounded up to whole warps); fewer threads
    // own several butterflies in the stages with more butterflies
    static constexpr int T = TT_ > 0 ? TT_ : ((N / SeqInfo<Fwd>::min_r) + 31) / 32 * 32;
    // shared memory (complex elements) of one transform: the larger padded
    // extent of the forward and the reversed chain, rounded up to an even
    // count so that staging areas placed after it start on a 16-byte
    // boundary (as cp.async of 16 bytes requires)
    static constexpr int SMEM_ELEMS = ((ChainExtent<Fwd>::value > ChainExtent<Inv>::value
                                            ? ChainExtent<Fwd>::value
                                            : ChainExtent<Inv>::value) + 1) / 2 * 2;
    static constexpr int SMEM_BYTES = 8 * SMEM_ELEMS;
    static_assert(T <= 1024, "too many threads per transform");
    using FwdChain = Chain<N, -1, 1, 0, T, Fwd>;
    using InvChain = Chain<N, +1, 1, 0, T, Inv>;
    // double-buffered chains: the inverse continues the forward's buffer
    // alternation (it follows the forward's exchanges in the column pass)
    static constexpr int NEX = SeqInfo<Fwd>::stages - 1;   // exchanges per chain
    using FwdChainDB = Chain<N, -1, 1, 0, T, Fwd, true, 0>;
    using InvChainDB = Chain<N, +1, 1, 0, T, Inv, true, NEX % 2>;
    static constexpr int E0 = FwdChain::E;                    // forward first stage
    static constexpr int EL = Chain<N, -1, N / RL, 0, T, Seq<RL>>::E;  // forward last stage
    static constexpr int EI = InvChain::E;                    // inverse first stage (= EL)
    static constexpr int EJ = Chain<N, +1, N / R0, 0, T, Seq<R0>>::E;  // inverse last stage
};

// Programmatic dependent launch.  The pass kernels are launched with the
// programmatic-stream-serialization attribute and begin with pdl_begin():
// the trigger lets the next kernel on the stream start launching once every
// block of this grid has started (its blocks then wait in their own
// pdl_begin), and the wait holds this grid until the previous grid on the
// stream has completed with its memory visible -- so no pass touches global
// memory before its predecessor is done, while the launch latency of each
// pass overlaps the tail of the one before.  Without the attribute (or after
// a non-kernel operation) the wait returns at once.  With LATE the block
// does not trigger, so the next kernel launches only as this grid's blocks
// exit: measured faster for the forward row pass at three resident blocks
// per SM (the next pass's early blocks otherwise share its last wave's SMs),
// a plan knob per pass.
template <bool LATE = false>
__device__ __forceinline__ void pdl_begin()
{
    if constexpr (!LATE) asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
}

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// P2's spectrum product on the forward column's last-stage outputs (thread
// t, butterfly j = t + e T holds frequencies j + m N/RL).
template <class P, int N, bool KREAL, bool STAGED>
__device__ __forceinline__ void spectrum_product(float2 (&f)[P::EL][P::RL], int t, const void* kcol,
                                                 const float* kst)
{
    constexpr int RL = P::RL, NBL = N / RL;
#pragma unroll
    for (int e = 0; e < P::EL; ++e) {
        const int j = t + e * P::T;
        if (j >= NBL) continue;
#pragma unroll
        for (int m = 0; m < RL; ++m) {
            const int u = j + m * NBL;
            if constexpr (KREAL) {
                const float k = STAGED ? kst[u] : __ldg(static_cast<const float*>(kcol) + u);
                f[e][m] = cscale(f[e][m], k);
            } else {
                const float2 k = STAGED ? reinterpret_cast<const float2*>(kst)[u]
                                        : __ldg(static_cast<const float2*>(kcol) + u);
                f[e][m] = cmul(f[e][m], k);
            }
        }
    }
}

// P2's inverse-output store: rows of the crop window of column Uc.
template <class P, int N>
__device__ __forceinline__ void store_column(const float2 (&o)[P::EJ][P::R0], int t, float2* Uc,
                                             int r0, int Hout, int HoutPad)
{
    constexpr int R0 = P::R0, NB0 = N / R0;
#pragma unroll
    for (int e = 0; e < P::EJ; ++e) {
        const int j = t + e * P::T;
        if (j >= NB0) continue;
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            int rr = j + m * NB0 - r0;
            if (rr < 0) rr += N;
            if (rr < Hout) Uc[u_row(rr)] = o[e][m];
        }
    }
    if (HoutPad != Hout && t == 0) Uc[u_row(Hout)] = make_float2(0.f, 0.f);
}

// P1's split of the packed transform Z (in shared memory, natural order)
// into the half spectra of rows a and b: {2 X_a[c], 2 X_b[c]} -> T[c][pair].
template <int N, int T>
__device__ __forceinline__ void unpack_rows(const float2* sm, int t, int ncols, float4* Tq, long long ldq,
                                            int pair)
{
    for (int c = t; c < ncols; c += T) {
        const int cm = (c == 0) ? 0 : N - c;
        const float2 zc = sm[c], zm = sm[cm];
        float4 o;
        o.x = zc.x + zm.x;       // 2 X_a = Z[c] + conj Z[N-c]
        o.y = zc.y - zm.y;
        o.z = zc.y + zm.y;       // 2 X_b = -i (Z[c] - conj Z[N-c])
        o.w = -(zc.x - zm.x);
        Tq[t_index4(c, pair, ldq)] = o;
    }
}

// P1/P3 hand the last stage's outputs to shared memory in natural order.
template <class P, int N, int E, int R>
__device__ __forceinline__ void to_smem_natural(const float2 (&z)[E][R], int t, float2* sm)
{
    constexpr int NBL = N / R;
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int j = t + e * P::T;
        if (j >= NBL) continue;
#pragma unroll
        for (int m = 0; m < R; ++m) sm[j + m * NBL] = z[e][m];
    }
    __syncthreads();
}

// P3's first-stage input: Z[k] = A[k] + i B[k] from the stored half spectra
// q = {A, B} of k (k <= N/2) or of N-k (Hermitian extension).
__device__ __forceinline__ float2 packed_inverse_input(float4 q, bool lo, bool vb)
{
    if (!vb) {
        q.z = 0.f;
        q.w = 0.f;
    }
    return lo ? make_float2(q.x - q.w, q.y + q.z) : make_float2(q.x + q.w, q.z - q.y);
}

// P3's final store: real part -> row a, imaginary part -> row b, crop columns.
template <class P, int N>
__device__ __forceinline__ void store_rows(const float2 (&o)[P::EJ][P::R0], int t, float* oa, float* ob,
                                           bool vb, int c0, int Wout)
{
    constexpr int RJ = P::R0, NBJ = N / RJ;
#pragma unroll
    for (int e = 0; e < P::EJ; ++e) {
        const int j = t + e * P::T;
        if (j >= NBJ) continue;
#pragma unroll
        for (int m = 0; m < RJ; ++m) {
            int cc = j + m * NBJ - c0;
            if (cc < 0) cc += N;
            if (cc < Wout) {
                oa[cc] = o[e][m].x;
                if (vb) ob[cc] = o[e][m].y;
            }
        }
    }
}

// ---------------------------------------------------------------------------
// P1: row R2C of two packed rows per transform, F transforms per block.
// ---------------------------------------------------------------------------
template <class P, int N, int F, bool LATE = false>
__global__ void __launch_bounds__(P::T * F) p1_rows(const P1Args a)
{
    pdl_begin<LATE>();
    extern __shared__ float2 smem2[];
    constexpr int T = P::T;
    constexpr int R0 = P::R0, NB0 = N / R0;
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    float2* sm = smem2 + f * P::SMEM_ELEMS;
    const int pair = a.pair0 + blockIdx.x * F + f;
    const int ra = 2 * pair, rb = ra + 1;
    const bool live = pair < a.npairs && p1_unit_ok(a, pair);
    const bool va = live && ra < a.H, vb = live && rb < a.H;
    const float* La = a.L + (long long)ra * a.ldl;
    const float* Lb = a.L + (long long)rb * a.ldl;

    float2 v[P::E0][R0];
#pragma unroll
    for (int e = 0; e < P::E0; ++e) {
        const int j = t + e * T;
        if (j >= NB0) continue;
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int col = j + m * NB0;
            const bool in = col < a.W;
            v[e][m].x = (in && va) ? __ldg(La + col) : 0.f;
            v[e][m].y = (in && vb) ? __ldg(Lb + col) : 0.f;
        }
    }
    P::FwdChain::run(v, t, sm, a.tw, [&](float2(&z)[P::EL][P::RL], int tt) {
        to_smem_natural<P, N>(z, tt, sm);
        if (live) unpack_rows<N, T>(sm, tt, a.ncols, reinterpret_cast<float4*>(a.T), a.ldT / 2, pair);
    });
}

// ---------------------------------------------------------------------------
// P2: per column forward FFT, spectrum product, inverse FFT, row crop.
// ---------------------------------------------------------------------------
// One spectrum of the batched column pass: the forward column is parked in
// F (natural order); product with spectrum s, inverse, store.  Not inlined:
// as a loop body it would let the compiler keep the whole inverse's
// constants and indices live across iterations.
template <class P, int N, bool KREAL>
__device__ __noinline__ void p2_spectrum_pass(const P2Args& a, int c, int s, const float2* F, float2* sm)
{
    constexpr int RL = P::RL, NBL = N / RL;
    const int t = threadIdx.x;
    float2 g[P::EL][RL];
#pragma unroll
    for (int e = 0; e < P::EL; ++e) {
        const int j = t + e * P::T;
        if (j >= NBL) continue;
#pragma unroll
        for (int m = 0; m < RL; ++m) g[e][m] = F[j + m * NBL];
    }
    const long long kw = KREAL ? 1 : 2;
    spectrum_product<P, N, KREAL, false>(g, t, static_cast<const float*>(a.K[s]) + (long long)c * a.ldK * kw,
                                         nullptr);
    float2* Uc = u_column(a.U + (long long)s * a.specU, a.ldU, c);
    P::InvChain::run(g, t, sm, a.twi, [&](float2(&o)[P::EJ][P::R0], int tt) {
        store_column<P, N>(o, tt, Uc, a.r0, a.Hout, a.HoutPad);
    });
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem);
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem);
// bulk prefetch of [p, p + bytes) into L2 (p 16-byte aligned, bytes a
// multiple of 16)
__device__ __forceinline__ void l2_prefetch(const void* p, unsigned bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit();
__device__ __forceinline__ void cp_async_wait_all();

// KST (one spectrum): the block's spectrum column is copied into shared
// memory (after the exchange buffer) with cp.async at the start, so its
// load latency overlaps the forward transform instead of stalling the
// product.
// PARKG (several spectra): the forward column is parked in global memory
// (a.park) instead of shared memory, for lengths whose exchange buffer and
// parked column do not fit shared memory together.
template <class P, int N, bool KREAL, bool MULTI, int MINB = 1, bool DB = false, bool KST = false,
          bool PARKG = false, bool LATE = false>
__global__ void __launch_bounds__(P::T, MINB) p2_cols(const __grid_constant__ P2Args a)
{
    pdl_begin<LATE>();
    static_assert(!(DB && MULTI), "the batched column pass is single-buffered");
    static_assert(!(KST && MULTI), "spectrum staging is for one spectrum");
    using Fwd = typename std::conditional<DB, typename P::FwdChainDB, typename P::FwdChain>::type;
    using Inv = typename std::conditional<DB, typename P::InvChainDB, typename P::InvChain>::type;
    extern __shared__ float2 smem2[];
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int RL = P::RL, NBL = N / RL;
    float2* sm = smem2;
    const int c = blockIdx.x;
    const int t = threadIdx.x;
    constexpr int KW = KREAL ? 1 : 2;  // floats per spectrum value
    if (!p2_column_ok(a, c, N, KW)) return;  // (whole block: before any barrier)
    const float2* col = t_column(a.T, a.ldT, c);
    float* kst = reinterpret_cast<float*>(smem2 + (DB ? 2 : 1) * P::SMEM_ELEMS);
    if constexpr (!MULTI && !KST) {
        // the spectrum column is needed after the forward transform: one bulk
        // prefetch into L2 now (no shared memory, no barrier) shortens its
        // load latency at the product
        if (t == 0) l2_prefetch(static_cast<const float*>(a.K[0]) + (long long)c * a.ldK * KW, 16u * ((N * KW + 3) / 4));
        // the T columns of a block that starts about one wave of resident
        // blocks later (a.ahead columns on), so that its first loads hit L2;
        // the even column of each pair prefetches the pair's block
        const int cn = c + a.ahead;
        if (t == 32 && a.ahead > 0 && (cn & 1) == 0 && cn < a.ncols)
            l2_prefetch(t_column(a.T, a.ldT, cn), (unsigned)(16 * a.ldT));
    }
    if constexpr (KST) {
        // ldK is a multiple of 32, so the column start is 16-byte aligned
        const float* src = static_cast<const float*>(a.K[0]) + (long long)c * a.ldK * KW;
        for (int q = t; q < (N * KW + 3) / 4; q += P::T) cp_async16(kst + 4 * q, src + 4 * q);
        cp_async_commit();
    }

    float2 v[P::E0][R0];
#pragma unroll
    for (int e = 0; e < P::E0; ++e) {
        const int j = t + e * P::T;
        if (j >= NB0) continue;
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int row = j + m * NB0;
            const long long off = (NB0 % 2 == 0) ? t_row(j) + m * t_row_step<NB0>() : t_row(row);
            v[e][m] = row < a.H ? __ldg(col + off) : make_float2(0.f, 0.f);
        }
    }
    Fwd::run(v, t, sm, a.twf, [&](float2(&fz)[P::EL][RL], int tt) {
        if constexpr (MULTI) {
            // parked forward column, in shared memory after the exchange
            // buffer, or in global memory (L2-resident while the block runs);
            // each thread reads back only the elements it wrote, so no
            // barrier orders the park
            float2* F = PARKG ? a.park + (size_t)c * N : smem2 + P::SMEM_ELEMS;
#pragma unroll
            for (int e = 0; e < P::EL; ++e) {
                const int j = tt + e * P::T;
                if (j >= NBL) continue;
#pragma unroll
                for (int m = 0; m < RL; ++m) F[j + m * NBL] = fz[e][m];
            }
            for (int s = 0; s < a.nspec; ++s) p2_spectrum_pass<P, N, KREAL>(a, c, s, F, sm);
        } else {
            if constexpr (KST) {
                cp_async_wait_all();
                __syncthreads();  // every thread's share of the column has landed
            }
            spectrum_product<P, N, KREAL, KST>(fz, tt, static_cast<const float*>(a.K[0]) + (long long)c * a.ldK * KW,
                                               kst);
            float2* Uc = u_column(a.U, a.ldU, c);
            Inv::run(fz, tt, sm, a.twi, [&](float2(&o)[P::EJ][R0], int t2) {
                store_column<P, N>(o, t2, Uc, a.r0, a.Hout, a.HoutPad);
            }, P::SMEM_ELEMS);
        }
    }, P::SMEM_ELEMS);
}

// ---------------------------------------------------------------------------
// P3: row C2R of two packed rows per transform, F transforms per block,
// blockIdx.y selects the spectrum.
// ---------------------------------------------------------------------------
template <class P, int N, int F>
__global__ void __launch_bounds__(P::T * F) p3_rows(const P3Args a)
{
    pdl_begin();
    extern __shared__ float2 smem2[];
    constexpr int T = P::T;
    constexpr int RI = P::RL, NBI = N / RI;
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    float2* sm = smem2 + f * P::SMEM_ELEMS;
    const int pair = a.pair0 + blockIdx.x * F + f;
    const int sidx = blockIdx.y;
    const int ra = 2 * pair, rb = ra + 1;
    const float4* Uq = reinterpret_cast<const float4*>(a.U + (long long)sidx * a.specU);
    const long long ldq = a.ldU / 2;
    const bool live = pair < a.npairs && p3_unit_ok(a, pair, sidx);
    const bool vb = rb < a.Hout;

    float2 v[P::EI][RI];
#pragma unroll
    for (int e = 0; e < P::EI; ++e) {
        const int j = t + e * T;
        if (j >= NBI) continue;
#pragma unroll
        for (int m = 0; m < RI; ++m) {
            const int k = j + m * NBI;
            const bool lo = k < a.ncols;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            if (live) q = __ldg(Uq + u_index4(lo ? k : N - k, pair, ldq));
            v[e][m] = packed_inverse_input(q, lo, vb);
        }
    }
    P::InvChain::run(v, t, sm, a.tw, [&](float2(&o)[P::EJ][P::R0], int tt) {
        if (live) {
            float* oa = a.out[sidx] + (long long)ra * a.ldo;
            store_rows<P, N>(o, tt, oa, oa + a.ldo, vb, a.c0, a.Wout);
        }
    });
}

// ---------------------------------------------------------------------------
// Prefetching variants.  Each block handles UPB work units (u, u + gridDim.x,
// ...); while it transforms one unit, the input of the next one is copied
// into a shared-memory staging area with cp.async (16-byte pieces where
// aligned), so global-memory latency overlaps the butterflies instead of
// stalling them.  cp.async.wait_group is a hardware wait: no spin loop is
// involved.  Units are unrolled at compile time: a loop back-edge makes the
// compiler keep about 70 more registers live per thread.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// staging bytes of the prefetching kernels (host and device agree on these)
__host__ __device__ constexpr long long p1_stage_bytes(int Wst) { return 8ll * Wst; }
__host__ __device__ constexpr long long p2_stage_bytes(long long ldT, long long ldK, bool kreal, bool kstage)
{
    return 8ll * ldT + (kstage ? (kreal ? 4ll : 8ll) * ldK : 0ll);
}
__host__ __device__ constexpr long long p3_stage_bytes(int ncols) { return 16ll * ncols; }

template <class P, int N, int UPB, int MINB, bool DB = false, bool LATE = false>
__global__ void __launch_bounds__(P::T, MINB) p1_rows_pf(const P1Args a)
{
    pdl_begin<LATE>();
    extern __shared__ float2 smem2[];
    constexpr int T = P::T;
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int NBUF = DB ? 2 : 1;
    using Fwd = typename std::conditional<DB, typename P::FwdChainDB, typename P::FwdChain>::type;
    float2* sm = smem2;
    float* st = reinterpret_cast<float*>(smem2 + NBUF * P::SMEM_ELEMS);  // rows a, b: 2 x Wst floats
    const int Wst = a.Wst;

    auto prefetch = [&](int pair) {
        if (pair >= a.npairs || !p1_unit_ok(a, pair)) return;
        const int t = threadIdx.x;
        for (int r = 0; r < 2; ++r) {
            const int row = 2 * pair + r;
            if (row >= a.H) continue;
            const float* src = a.L + (long long)row * a.ldl;
            float* dst = st + r * Wst;
            if (a.vec16) {
                for (int q = t; q < (a.W >> 2); q += T) cp_async16(dst + 4 * q, src + 4 * q);
            } else {
                for (int i = t; i < a.W; i += T) cp_async4(dst + i, src + i);
            }
        }
        cp_async_commit();
    };
    auto unit = [&](int pair) {
        cp_async_wait_all();
        __syncthreads();
        const int t = threadIdx.x;
        const bool vb = 2 * pair + 1 < a.H;
        float2 v[P::E0][R0];
#pragma unroll
        for (int e = 0; e < P::E0; ++e) {
            const int j = t + e * T;
            if (j >= NB0) continue;
#pragma unroll
            for (int m = 0; m < R0; ++m) {
                const int col = j + m * NB0;
                const bool in = col < a.W;
                v[e][m].x = in ? st[col] : 0.f;
                v[e][m].y = (in && vb) ? st[Wst + col] : 0.f;
            }
        }
        __syncthreads();  // staging consumed
        prefetch(pair + gridDim.x);
        Fwd::run(v, t, sm, a.tw, [&](float2(&z)[P::EL][P::RL], int tt) {
            to_smem_natural<P, N>(z, tt, sm);
            unpack_rows<N, T>(sm, tt, a.ncols, reinterpret_cast<float4*>(a.T), a.ldT / 2, pair);
        }, P::SMEM_ELEMS);
    };
    prefetch(a.pair0 + blockIdx.x);
    sfor<0, UPB>([&](auto I) {
        const int pair = a.pair0 + blockIdx.x + decltype(I)::value * gridDim.x;
        if (pair < a.npairs && p1_unit_ok(a, pair)) unit(pair);
    });
}

// single spectrum; T column staged, K^ column staged when KSTAGE (else read
// directly at the product)
template <class P, int N, bool KREAL, int UPB, int MINB, bool KSTAGE, bool DB = false, bool LATE = false>
__global__ void __launch_bounds__(P::T, MINB) p2_cols_pf(const P2Args a)
{
    pdl_begin<LATE>();
    extern __shared__ float2 smem2[];
    constexpr int T = P::T;
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int RL = P::RL;
    constexpr int KW = KREAL ? 1 : 2;                    // floats per K^ element
    constexpr int NBUF = DB ? 2 : 1;
    using Fwd = typename std::conditional<DB, typename P::FwdChainDB, typename P::FwdChain>::type;
    using Inv = typename std::conditional<DB, typename P::InvChainDB, typename P::InvChain>::type;
    float2* sm = smem2;
    float2* tst = smem2 + NBUF * P::SMEM_ELEMS;          // ldT complex
    float* kst = reinterpret_cast<float*>(tst + a.ldT);  // ldK floats or complex

    auto prefetch_t = [&](int c) {
        if (c >= a.ncols || !p2_column_ok(a, c, N, KW)) return;
        const float4* src = reinterpret_cast<const float4*>(a.T);
        const long long ldq = a.ldT >> 1;
        for (int q = threadIdx.x; q < (int)ldq; q += T) cp_async16(tst + 2 * q, src + t_index4(c, q, ldq));
        cp_async_commit();
    };
    auto prefetch_k = [&](int c) {
        if constexpr (!KSTAGE) return;
        if (c >= a.ncols || !p2_column_ok(a, c, N, KW)) return;
        const float* src = static_cast<const float*>(a.K[0]) + (long long)c * a.ldK * KW;
        for (int q = threadIdx.x; q < (int)((a.ldK * KW) >> 2); q += T) cp_async16(kst + 4 * q, src + 4 * q);
        cp_async_commit();
    };

    auto unit = [&](int c) {
        cp_async_wait_all();
        __syncthreads();
        const int t = threadIdx.x;
        float2 v[P::E0][R0];
#pragma unroll
        for (int e = 0; e < P::E0; ++e) {
            const int j = t + e * T;
            if (j >= NB0) continue;
#pragma unroll
            for (int m = 0; m < R0; ++m) {
                const int row = j + m * NB0;
                v[e][m] = row < a.H ? tst[row] : make_float2(0.f, 0.f);
            }
        }
        __syncthreads();
        prefetch_t(c + gridDim.x);
        Fwd::run(v, t, sm, a.twf, [&](float2(&fz)[P::EL][RL], int tt) {
            spectrum_product<P, N, KREAL, KSTAGE>(
                fz, tt, static_cast<const float*>(a.K[0]) + (long long)c * a.ldK * KW, kst);
            if constexpr (KSTAGE) {
                __syncthreads();  // K^ staging consumed
                prefetch_k(c + gridDim.x);
            }
            float2* Uc = u_column(a.U, a.ldU, c);
            Inv::run(fz, tt, sm, a.twi, [&](float2(&o)[P::EJ][R0], int t2) {
                store_column<P, N>(o, t2, Uc, a.r0, a.Hout, a.HoutPad);
            }, P::SMEM_ELEMS);
        }, P::SMEM_ELEMS);
    };
    prefetch_t(blockIdx.x);
    prefetch_k(blockIdx.x);
    sfor<0, UPB>([&](auto I) {
        const int c = blockIdx.x + decltype(I)::value * gridDim.x;
        if (c < a.ncols && p2_column_ok(a, c, N, KW)) unit(c);
    });
}

template <class P, int N, int UPB, int MINB, bool DB = false>
__global__ void __launch_bounds__(P::T, MINB) p3_rows_pf(const P3Args a)
{
    pdl_begin();
    extern __shared__ float2 smem2[];
    constexpr int T = P::T;
    constexpr int RI = P::RL, NBI = N / RI;
    constexpr int NBUF = DB ? 2 : 1;
    using Inv = typename std::conditional<DB, typename P::InvChainDB, typename P::InvChain>::type;
    float2* sm = smem2;
    float4* ust = reinterpret_cast<float4*>(smem2 + NBUF * P::SMEM_ELEMS);  // ncols x {A, B}
    const int sidx = blockIdx.y;
    const float4* Uq = reinterpret_cast<const float4*>(a.U + (long long)sidx * a.specU);
    const long long ldq = a.ldU / 2;

    auto prefetch = [&](int pair) {
        if (pair >= a.npairs || !p3_unit_ok(a, pair, sidx)) return;
        for (int k = threadIdx.x; k < a.ncols; k += T) cp_async16(ust + k, Uq + u_index4(k, pair, ldq));
        cp_async_commit();
    };

    auto unit = [&](int pair) {
        cp_async_wait_all();
        __syncthreads();
        const int t = threadIdx.x;
        const int ra = 2 * pair, rb = ra + 1;
        const bool vb = rb < a.Hout;
        float2 v[P::EI][RI];
#pragma unroll
        for (int e = 0; e < P::EI; ++e) {
            const int j = t + e * T;
            if (j >= NBI) continue;
#pragma unroll
            for (int m = 0; m < RI; ++m) {
                const int k = j + m * NBI;
                const bool lo = k < a.ncols;
                v[e][m] = packed_inverse_input(ust[lo ? k : N - k], lo, vb);
            }
        }
        __syncthreads();
        prefetch(pair + gridDim.x);
        Inv::run(v, t, sm, a.tw, [&](float2(&o)[P::EJ][P::R0], int tt) {
            float* oa = a.out[sidx] + (long long)ra * a.ldo;
            store_rows<P, N>(o, tt, oa, oa + a.ldo, vb, a.c0, a.Wout);
        }, P::SMEM_ELEMS);
    };
    prefetch(a.pair0 + blockIdx.x);
    sfor<0, UPB>([&](auto I) {
        const int pair = a.pair0 + blockIdx.x + decltype(I)::value * gridDim.x;
        if (pair < a.npairs && p3_unit_ok(a, pair, sidx)) unit(pair);
    });
}

// ---------------------------------------------------------------------------
// P2 for Sec. 2.2 Eq. (4): several source classes, one PSF each.  The
// forward column transform of each class's T is multiplied by its spectrum
// and accumulated; one inverse transform follows.
// ---------------------------------------------------------------------------
struct P2MArgs {
    const float2* T[kMaxSpectraPerLaunch];
    long long ldT;
    int H;
    const void* K[kMaxSpectraPerLaunch];
    long long ldK;
    int nclass;
    float2* U;
    long long ldU;
    int r0, Hout, HoutPad;
    int ncols;
    TwChain twf, twi;
    float2* acc;  // the sums of the products, N per column (global memory)
    int* err;             // device status word (debug builds: bounds checks)
    long long t_elems;    // float2 elements of each class's T buffer
    long long k_elems;    // spectrum values of each spectrum
    long long u_elems;    // float2 elements of U
    long long acc_elems;  // float2 elements of the sums
};

// multiclass unit: column c of every class's T, of every spectrum, of U and of the sums
__device__ __forceinline__ bool p2m_column_ok(const P2MArgs& a, int c, int n)
{
#if LP_DEBUG
    return lp_checked(a.err, c >= 0 && c < a.ncols && a.H <= a.ldT && n <= a.ldK && a.HoutPad <= a.ldU &&
                                 2 * t_index4(c, 0, a.ldT / 2) + t_row((int)a.ldT - 1) < a.t_elems &&
                                 (long long)(c + 1) * a.ldK <= a.k_elems &&
                                 2 * u_index4(c, 0, a.ldU / 2) + u_row(a.HoutPad - 1) < a.u_elems &&
                                 (long long)(c + 1) * n <= a.acc_elems);
#else
    (void)a;
    (void)c;
    (void)n;
    return true;
#endif
}

// One class of the Eq. (4) column pass: forward transform of the class's
// column, product with its spectrum, summed into ACC (natural order; the
// first class writes it).  Each thread adds only to the elements it owns
// (j + m N/RL), so the sum needs no barrier.  Not inlined, for the same
// reason as p2_spectrum_pass.
template <class P, int N, bool KREAL>
__device__ __noinline__ void p2_class_pass(const P2MArgs& a, int c, int q, float2* ACC, float2* sm)
{
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int RL = P::RL, NBL = N / RL;
    const int t = threadIdx.x;
    const float2* col = t_column(a.T[q], a.ldT, c);
    float2 v[P::E0][R0];
#pragma unroll
    for (int e = 0; e < P::E0; ++e) {
        const int j = t + e * P::T;
        if (j >= NB0) continue;
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int row = j + m * NB0;
            const long long off = (NB0 % 2 == 0) ? t_row(j) + m * t_row_step<NB0>() : t_row(row);
            v[e][m] = row < a.H ? __ldg(col + off) : make_float2(0.f, 0.f);
        }
    }
    P::FwdChain::run(v, t, sm, a.twf, [&](float2(&fz)[P::EL][RL], int tt) {
        const long long kw = KREAL ? 1 : 2;
        spectrum_product<P, N, KREAL, false>(fz, tt, static_cast<const float*>(a.K[q]) + (long long)c * a.ldK * kw,
                                             nullptr);
#pragma unroll
        for (int e = 0; e < P::EL; ++e) {
            const int j = tt + e * P::T;
            if (j >= NBL) continue;
#pragma unroll
            for (int m = 0; m < RL; ++m) {
                float2& acc = ACC[j + m * NBL];
                acc = q == 0 ? fz[e][m] : cadd(acc, fz[e][m]);
            }
        }
    });
}

template <class P, int N, bool KREAL>
__global__ void __launch_bounds__(P::T) p2_multiclass(const __grid_constant__ P2MArgs a)
{
    pdl_begin();
    extern __shared__ float2 smem2[];
    constexpr int RL = P::RL, NBL = N / RL;
    float2* sm = smem2;
    const int c = blockIdx.x;
    const int t = threadIdx.x;
    if (!p2m_column_ok(a, c, N)) return;  // (whole block: before any barrier)
    // the sums live in global memory (L2-resident while the block runs), so
    // shared memory holds one exchange buffer at every length; every
    // element of ACC is owned by one thread (j + m N/RL), which writes it for
    // the first class, adds to it for the others and reads it back below
    float2* ACC = a.acc + (size_t)c * N;
    for (int q = 0; q < a.nclass; ++q) p2_class_pass<P, N, KREAL>(a, c, q, ACC, sm);
    float2 acc[P::EL][RL];
#pragma unroll
    for (int e = 0; e < P::EL; ++e) {
        const int j = t + e * P::T;
        if (j >= NBL) continue;
#pragma unroll
        for (int m = 0; m < RL; ++m) acc[e][m] = ACC[j + m * NBL];
    }
    float2* Uc = u_column(a.U, a.ldU, c);
    P::InvChain::run(acc, t, sm, a.twi, [&](float2(&o)[P::EJ][P::R0], int tt) {
        store_column<P, N>(o, tt, Uc, a.r0, a.Hout, a.HoutPad);
    });
}

}  // namespace lpk
