// Column pass with the DFT stages on the tensor cores (split BF16, FP32
// accumulation): the LP_PREC_SPLIT_BF16 form of P2.
//
// A radix-R stage of the Stockham chain (see fft_core.cuh) is, for each of
// its NB = N/R butterflies, y = F_R x with F_R the R-point DFT matrix of
// Sec. 2.3 Eq. (10).  In real form y (2R reals: Re, Im interleaved) is a
// 2R x 2R matrix times x, so one stage of all butterflies of a column is the
// GEMM  D[NB x 2R] = A[NB x 2R] * F^T  with A holding one butterfly's
// twiddled inputs per row.  Each operand is split into BF16 hi + lo parts
// (x = x_hi + x_lo to about 2^-16), and D = A_hi F_hi + A_hi F_lo + A_lo F_hi
// is accumulated in FP32 by tcgen05.mma into tensor memory (TMEM).
//
// Data flow of one stage: every thread reads its butterfly's row of D from
// TMEM, and writes each output straight into the next stage's A operand at
// the row and column the Stockham order gives it, after applying the next
// stage's twiddle and splitting it into hi/lo -- so no FP32 exchange buffer
// is needed.  Between the forward and the inverse column transform the
// outputs are multiplied by the PSF spectrum; after the inverse, the kept
// rows are stored to U.  The inverse runs as conj(DFT(conj(x))), so both
// chains use the forward matrices and twiddle signs.  The row passes P1 and
// P3 stay in FP32.
//
// Shared-memory operand layout (the canonical "no swizzle, K-major" form):
// 8 x 16-byte core matrices, core (row group g, k group kg) at byte
// ((g * KG) + kg) * 128 within a 128-row tile (KG = Kp / 8); descriptors use
// leading byte offset 128 (next k group) and stride byte offset KG * 128
// (next row group).  Every wait on the MMA's mbarrier is bounded; on time-out
// the kernel sets bit 2 of the device status word and stops.
#pragma once

#include <cuda_bf16.h>

#include "conv_kernels.cuh"

namespace lpk {

constexpr int ru16(int x) { return (x + 15) / 16 * 16; }

// Tables of the pass, one contiguous device block copied to shared memory
// by every block: the forward DFT matrices of the forward chain's stages --
// per stage hi then lo, each Kp x Kp bf16 in the core-matrix layout (rows =
// outputs n, columns = inputs k, zero padded) -- then the twiddle step
// factors of the forward and of the reversed chain: per stage s >= 1,
// exp(-i 2 pi m k / (R_{s-1} R_s)) at [m R_{s-1} + k], m < R_s, k < R_{s-1}.
// The inverse transform runs as conj(DFT(conj(x))) on the same matrices.
struct P2TcArgs {
    P2Args a;  // as the FP32 column pass, one spectrum (a.K[0])
    const uint4* tables;
    int* err;  // device status word (bit 2: an MMA wait timed out)
    int no_mma;  // test hook: issue no MMA, so the first bounded wait runs out
};

__device__ __forceinline__ uint32_t sm_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// The pass's dynamic shared memory, A operand at offset 0.  Declared at
// namespace scope so that the non-inlined column body addresses it as
// shared memory (32-bit addresses) rather than through generic pointers.
extern __shared__ __align__(1024) unsigned char tc_dsmem[];

__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of this architecture; no swizzle
    return d;
}

// byte offset of element (r, k) of a 128-row tile with KG k-groups
__device__ __forceinline__ uint32_t tc_off(int r, int k, int KG)
{
    return (uint32_t)((((r >> 3) * KG + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// hi/lo BF16 pairs of a complex value
__device__ __forceinline__ void tc_split(float2 z, uint32_t& hi, uint32_t& lo)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(z.x, z.y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(z.x - hf.x, z.y - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

// Geometry of one stage (radix R, group size Ns) of a length-N chain.
template <int N, int R_, int Ns_>
struct TcStage {
    static constexpr int R = R_;
    static constexpr int Ns = Ns_;
    static constexpr int NB = N / R;
    static constexpr int KP = ru16(2 * R);               // padded K (= N of the MMA)
    static constexpr int KG = KP / 8;
    static constexpr int TILES = (NB + 127) / 128;
    static constexpr int TILE_BYTES = 128 * KP * 2;      // one of hi / lo
    static constexpr int MAT_BYTES = 2 * KP * KP * 2;    // hi + lo
};

template <int N, class S> struct TcChainInfo;
template <int N, int... Rs> struct TcChainInfo<N, Seq<Rs...>> {
    static constexpr int S = sizeof...(Rs);
    static constexpr int a_bytes()
    {
        const int rs[] = {Rs...};
        int m = 0;
        for (int s = 0; s < S; ++s) {
            const int nb = N / rs[s], kp = ru16(2 * rs[s]);
            const int b = 2 * ((nb + 127) / 128) * 128 * kp * 2;
            m = b > m ? b : m;
        }
        return m;
    }
    // bytes of the matrices of stages [0, upto)
    static constexpr int mat_bytes(int upto = S)
    {
        const int rs[] = {Rs...};
        int t = 0;
        for (int s = 0; s < upto; ++s) t += 2 * ru16(2 * rs[s]) * ru16(2 * rs[s]) * 2;
        return t;
    }
    // bytes of the step factors of stages [1, upto)
    static constexpr int step_bytes_upto(int upto)
    {
        const int rs[] = {Rs...};
        int b = 0;
        for (int s = 1; s < upto; ++s) b += rs[s - 1] * rs[s] * 8;
        return b;
    }
    static constexpr int step_bytes()
    {
        const int rs[] = {Rs...};
        int b = 0;
        for (int s = 1; s < S; ++s) b += rs[s - 1] * rs[s] * 8;
        return b;
    }
    static constexpr int tmem_cols()
    {
        const int rs[] = {Rs...};
        int m = 0;
        for (int s = 0; s < S; ++s) {
            const int c = ((N / rs[s] + 127) / 128) * ru16(2 * rs[s]);
            m = c > m ? c : m;
        }
        int p = 32;
        while (p < m) p *= 2;
        return p;
    }
};

// threads of the tensor-core column pass: one per butterfly of the stage
// with the most butterflies, whole warps
template <class P, int N>
constexpr int tc_threads()
{
    return ((N / SeqInfo<typename P::Fwd>::min_r) + 31) / 32 * 32;
}

template <class P, int N>
struct TcPlan {
    using FI = TcChainInfo<N, typename P::Fwd>;
    using II = TcChainInfo<N, typename P::Inv>;
    static constexpr int S = FI::S;
    static constexpr int A_BYTES = FI::a_bytes();   // the inverse has the same radices
    // one matrix per forward stage: the inverse chain runs in the conjugate
    // domain on the same (forward) matrices
    static constexpr int MAT_BYTES = FI::mat_bytes();
    static constexpr int STEPF_BYTES = FI::step_bytes();
    static constexpr int TAB_BYTES = (MAT_BYTES + STEPF_BYTES + II::step_bytes() + 15) / 16 * 16;
    static constexpr int TMEM_COLS = FI::tmem_cols();
    static constexpr int SMEM_BYTES = A_BYTES + TAB_BYTES + 64;
    static constexpr int THREADS = tc_threads<P, N>();
    static constexpr bool FITS = TMEM_COLS <= 512 && SMEM_BYTES <= 227 * 1024 && THREADS <= 1024;
    // resident blocks per SM for the launch bounds' register budget: what
    // the shared memory allows, at most 3, and no more than leaves 56
    // registers per thread
    static constexpr int BY_SMEM = (228 * 1024) / (SMEM_BYTES + 1024);
    static constexpr int BY_REGS = 65536 / (THREADS * 56);
    static constexpr int MINB_ = BY_SMEM < BY_REGS ? BY_SMEM : BY_REGS;
    static constexpr int MINB = MINB_ < 1 ? 1 : (MINB_ > 3 ? 3 : MINB_);
    // shared-memory layout of the stages: matrix byte offset (from the
    // matrices' base) and step-factor byte offset (from the dynamic shared
    // memory's base); inverse stage s uses forward stage S-1-s's matrix
    struct FwdLayout {
        static constexpr int moff(int s) { return FI::mat_bytes(s); }
        static constexpr int soff(int s) { return A_BYTES + MAT_BYTES + FI::step_bytes_upto(s + 1); }
    };
    struct InvLayout {
        static constexpr int moff(int s) { return FI::mat_bytes(S - 1 - s); }
        static constexpr int soff(int s) { return A_BYTES + MAT_BYTES + STEPF_BYTES + II::step_bytes_upto(s + 1); }
    };
};

// Issue the split-precision MMAs of one stage (one thread) and commit them
// to the mbarrier: D = A_hi B_hi + A_hi B_lo + A_lo B_hi per 128-row tile.
template <class G>
__device__ __forceinline__ void tc_issue(uint32_t tbase, uint32_t a_smem, uint32_t b_smem, uint32_t mbar)
{
    // opaque operands: keeps the (loop-invariant) descriptors of every stage
    // from being hoisted out of the column loop into registers
    asm volatile("" : "+r"(tbase), "+r"(a_smem), "+r"(b_smem));
    constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(G::KP >> 3) << 17) |
                               ((uint32_t)(128 >> 4) << 24);
    constexpr uint32_t lbo = 128, sbo = G::KG * 128;
#pragma unroll
    for (int m = 0; m < G::TILES; ++m) {
        const uint32_t d = tbase + (uint32_t)(m * G::KP);
        const uint32_t ahi = a_smem + m * G::TILE_BYTES;
        const uint32_t alo = a_smem + (G::TILES + m) * G::TILE_BYTES;
        const uint32_t bhi = b_smem, blo = b_smem + G::KP * G::KP * 2;
#pragma unroll
        for (int s = 0; s < G::KP / 16; ++s) {
            const uint64_t dah = tc_sdesc(ahi + s * 256, lbo, sbo), dal = tc_sdesc(alo + s * 256, lbo, sbo);
            const uint64_t dbh = tc_sdesc(bhi + s * 256, lbo, sbo), dbl = tc_sdesc(blo + s * 256, lbo, sbo);
            const uint32_t acc = s > 0 ? 1u : 0u;
            asm volatile(
                "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %5, %3, 1;\n"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %6, %2, %3, 1;\n}\n" ::"r"(d),
                "l"(dah), "l"(dbh), "r"(idesc), "r"(acc), "l"(dbl), "l"(dal));
        }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ uint64_t tc_globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
    return t;
}

// Bounded wait for one phase of the MMA mbarrier: gives up after 100 ms of
// device time (an MMA round trip takes microseconds), with an iteration cap
// behind it.
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t phase)
{
    uint32_t done = 0;
    const uint64_t t0 = tc_globaltimer();
    for (int it = 0; it < (1 << 24) && !done; ++it) {
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(mbar), "r"(phase)
            : "memory");
        if (!done && (it & 63) == 63 && tc_globaltimer() - t0 > 100000000ull) break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    return done != 0;
}

// Read 16 columns (8 complex outputs, from output c0 / 2 on) of this
// thread's butterfly row of D from TMEM.  Warp-collective: warp w reaches
// TMEM lanes 32 (w mod 4) .. +31, i.e. rows of tile w / 4; warps past the
// last tile do not load.
template <class G>
__device__ __forceinline__ void tc_read8(uint32_t tbase, int c0, float2 (&y)[8])
{
    const int w = threadIdx.x >> 5;
    const int m = w >> 2;
    if (m >= G::TILES) return;
    const uint32_t ta = tbase + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(m * G::KP + c0);
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(ta));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) y[i] = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
}

// Write z (split hi/lo) into the A operand of stage G at row j, input slot q.
template <class G>
__device__ __forceinline__ void tc_put(int j, int q, float2 z)
{
    unsigned char* As = tc_dsmem;
    uint32_t hi, lo;
    tc_split(z, hi, lo);
    const uint32_t off = (uint32_t)((j >> 7) * G::TILE_BYTES) + tc_off(j & 127, 2 * q, G::KG);
    *reinterpret_cast<uint32_t*>(As + off) = hi;
    *reinterpret_cast<uint32_t*>(As + off + G::TILES * G::TILE_BYTES) = lo;
}

// zero the padding inputs [R, KP/2) of row j of stage G (hi and lo)
template <class G>
__device__ __forceinline__ void tc_zero_pad(int j)
{
    unsigned char* As = tc_dsmem;
#pragma unroll
    for (int q = G::R; q < G::KP / 2; ++q) {
        const uint32_t off = (uint32_t)((j >> 7) * G::TILE_BYTES) + tc_off(j & 127, 2 * q, G::KG);
        *reinterpret_cast<uint32_t*>(As + off) = 0u;
        *reinterpret_cast<uint32_t*>(As + off + G::TILES * G::TILE_BYTES) = 0u;
    }
}

// Per-block state of the tensor-core column pass.
struct TcState {
    int no_mma;           // test hook (see P2TcArgs)
    uint32_t bsm;         // shared address of the DFT matrices
    uint32_t tbase;       // TMEM base
    uint32_t mbar;        // shared address of the MMA mbarrier
    uint32_t phase;
    int* dead;            // shared flag: an MMA wait timed out
};

// One chain of tensor-core stages.  Precondition: the A operand holds the
// first stage's twiddled inputs (rows = butterflies).  Every thread of the
// block calls `run` (it contains barriers).  The last stage's outputs go to
// `sink(k, z)`: output t + k N/R_last of the chain (the last stage's
// butterfly t), called only where thread t owns such a butterfly and every
// MMA completed.  Outputs are consumed 8 at a time as they leave TMEM;
// `sink.pad()` runs first, after the last MMA wait (the sink's own writes
// of the A operand start there).
template <int N, int Ns, int SIdx, class LO, class S> struct TcChain;

template <int N, int Ns, int SIdx, class LO, int R, int... Rest>
struct TcChain<N, Ns, SIdx, LO, Seq<R, Rest...>> {
    using G = TcStage<N, R, Ns>;

    // issue this stage's MMAs and wait for them; false if the block is dead
    __device__ __forceinline__ static bool mma(TcState& st, int* err)
    {
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        const bool dead = *st.dead != 0;
        if (!dead && threadIdx.x == 0 && !st.no_mma) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            tc_issue<G>(st.tbase, sm_u32(tc_dsmem), st.bsm + LO::moff(SIdx), st.mbar);
        }
        bool ok = dead ? false : tc_wait(st.mbar, st.phase);
        st.phase ^= 1u;
        if (!dead && !ok) {
            *st.dead = 1;
            atomicOr(err, 4);
        }
        return __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
    }

    template <class Sink>
    __device__ __forceinline__ static void run(TcState& st, const TwChain& tw, int* err, int t, Sink& sink)
    {
        if constexpr (sizeof...(Rest) == 0) {
            sink.prefetch();  // global loads of the sink overlap the last MMA
            const bool ok = mma(st, err);
            sink.pad();
            if (ok) {
#pragma unroll
                for (int c0 = 0; c0 < G::KP; c0 += 16) {
                    float2 y[8];
                    tc_read8<G>(st.tbase, c0, y);
                    if (t < G::NB) {
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (c0 / 2 + i < R) sink(c0 / 2 + i, y[i]);
                    }
                }
            }
        } else {
            constexpr int R2 = SeqInfo<Seq<Rest...>>::first;
            using G2 = TcStage<N, R2, Ns * R>;
            // Stockham placement: output k of butterfly t goes to
            // p = (t / Ns) P + t mod Ns + k Ns (P = Ns R).  The next stage's
            // butterfly count NB2 is a multiple of P, so its slot m2 = p / NB2
            // is the same for every k and its butterfly is j2 = j20 + k Ns.
            // Its twiddle exp(-i 2 pi m2 (t mod Ns + k Ns) / (P R2)) is w0
            // (the table entry of k = 0, loaded before the MMA wait) times
            // the step factor exp(-i 2 pi m2 k / (R R2)) (shared table).
            constexpr int P = Ns * R;
            static_assert(G2::NB % P == 0, "next stage's butterfly count must be a multiple of the group size");
            const int base = (t / Ns) * P + (t % Ns);
            const int m2 = base / G2::NB;
            const int j20 = base - m2 * G2::NB;
            const float2* tab = tw.p[SIdx + 1];
            asm volatile("" : "+l"(tab));  // no hoisting above the previous stage's wait
            float2 w0 = make_float2(1.f, 0.f);
            if (m2 > 0 && t < G::NB) w0 = __ldg(tab + (m2 - 1) * P + (t % Ns));
            const bool ok = mma(st, err);
            if (t < G2::NB) tc_zero_pad<G2>(t);
            if (ok) {
                const float2* step = reinterpret_cast<const float2*>(tc_dsmem + LO::soff(SIdx)) + m2 * R;
#pragma unroll
                for (int c0 = 0; c0 < G::KP; c0 += 16) {
                    float2 y[8];
                    tc_read8<G>(st.tbase, c0, y);
                    if (t < G::NB) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const int k = c0 / 2 + i;
                            if (k >= R) continue;
                            float2 z = y[i];
                            if (m2 > 0) z = cmul(z, cmul(w0, step[k]));
                            tc_put<G2>(j20 + k * Ns, m2, z);
                        }
                    }
                }
            }
            TcChain<N, Ns * R, SIdx + 1, LO, Seq<Rest...>>::run(st, tw, err, t, sink);
        }
    }
};

// Sinks of the two chains of the column pass.
// Forward: product with the PSF spectrum at frequency t + k N/RL; the
// products are the first inverse stage's inputs (butterfly t, slot k, no
// twiddle).
template <int N, int RL, bool KREAL, class GI0>
struct TcProductSink {
    const void* kcol;  // spectrum column c
    int t;
    typename std::conditional<KREAL, float, float2>::type kv[RL];
    // before the forward chain's last MMA wait: the spectrum values of this
    // thread's frequencies (the pointer becomes opaque here, so the loads are
    // not hoisted further up)
    __device__ __forceinline__ void prefetch()
    {
        asm volatile("" : "+l"(kcol));
        if (t < N / RL) {
#pragma unroll
            for (int k = 0; k < RL; ++k) {
                const int f = t + k * (N / RL);
                if constexpr (KREAL) kv[k] = __ldg(static_cast<const float*>(kcol) + f);
                else kv[k] = __ldg(static_cast<const float2*>(kcol) + f);
            }
        }
    }
    // after the last MMA wait: the A operand now takes the inverse's inputs
    __device__ __forceinline__ void pad()
    {
        if (t < GI0::NB) tc_zero_pad<GI0>(t);
    }
    __device__ __forceinline__ void operator()(int k, float2 z) const
    {
        if constexpr (KREAL) z = make_float2(z.x * kv[k], z.y * kv[k]);
        else z = cmul(z, kv[k]);
        tc_put<GI0>(t, k, make_float2(z.x, -z.y));  // the inverse runs on conjugates
    }
};

// Inverse: output row t + k N/R0 of the circular result, kept rows to U.
template <int N, int R0>
struct TcStoreSink {
    float2* Uc;
    int r0, Hout, t;
    __device__ __forceinline__ void prefetch() {}
    __device__ __forceinline__ void pad() {}
    __device__ __forceinline__ void operator()(int k, float2 z) const
    {
        int rr = t + k * (N / R0) - r0;
        if (rr < 0) rr += N;
        if (rr < Hout) Uc[u_row(rr)] = make_float2(z.x, -z.y);  // back from the conjugate domain
    }
};

// One column c of one spectrum: forward column DFT, spectrum product,
// inverse, crop.  Not inlined: as the body of the persistent loop the
// compiler keeps more state live across the loop's back edge and spills at
// the register budget of two resident blocks per SM.
template <class P, int N, bool KREAL>
__device__ __noinline__ void tc_column(const P2TcArgs& A, int c, TcState& st)
{
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int RL = P::RL;
    using TP = TcPlan<P, N>;
    using G0 = TcStage<N, R0, 1>;   // first forward stage
    using GI0 = TcStage<N, RL, 1>;  // first inverse stage
    using Fwd = TcChain<N, 1, 0, typename TP::FwdLayout, typename P::Fwd>;
    // the inverse transform as conj(DFT(conj(x))): the same forward matrices,
    // step factors and twiddle signs; the product sink stores conjugates and
    // the store sink conjugates back
    using Inv = TcChain<N, 1, 0, typename TP::InvLayout, typename P::Inv>;
    const P2Args& a = A.a;
    const int t = threadIdx.x;
    __syncthreads();  // the previous column's last writes of As are consumed
    // first forward stage: rows j + m N/R0 of column c (rows >= H are the zero padding)
    if (t < NB0) {
        const float2* col = t_column(a.T, a.ldT, c);
        tc_zero_pad<G0>(t);
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int row = t + m * NB0;
            const long long off = (NB0 % 2 == 0) ? t_row(t) + m * t_row_step<NB0>() : t_row(row);
            tc_put<G0>(t, m, row < a.H ? __ldg(col + off) : make_float2(0.f, 0.f));
        }
    }
    {
        const void* kcol = static_cast<const char*>(a.K[0]) + (long long)c * a.ldK * (KREAL ? 4 : 8);
        TcProductSink<N, RL, KREAL, GI0> ps{kcol, t};
        Fwd::run(st, a.twf, A.err, t, ps);
    }
    float2* Uc = u_column(a.U, a.ldU, c);
    TcStoreSink<N, R0> ss{Uc, a.r0, a.Hout, t};
    Inv::run(st, a.twi, A.err, t, ss);
    if (a.HoutPad != a.Hout && t == 0) Uc[u_row(a.Hout)] = make_float2(0.f, 0.f);
}

// The column pass: persistent blocks, one column of one spectrum at a time.
template <class P, int N, bool KREAL>
__global__ void __launch_bounds__(TcPlan<P, N>::THREADS, TcPlan<P, N>::MINB) p2_cols_tc(const __grid_constant__ P2TcArgs A)
{
    pdl_begin();
    using TP = TcPlan<P, N>;
    const P2Args& a = A.a;
    const int t = threadIdx.x;
    unsigned char* Bs = tc_dsmem + TP::A_BYTES;
    uint64_t* mbar = reinterpret_cast<uint64_t*>(Bs + TP::TAB_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    int* dead = reinterpret_cast<int*>(tslot + 1);

    // matrices and step factors into shared memory
    {
        uint4* dst = reinterpret_cast<uint4*>(Bs);
        for (int i = t; i < TP::TAB_BYTES / 16; i += blockDim.x) dst[i] = A.tables[i];
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sm_u32(mbar)));
        *dead = 0;
    }
    if (t < 32) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sm_u32(tslot)),
                     "r"(TP::TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    TcState st{A.no_mma, sm_u32(Bs), *tslot, sm_u32(mbar), 0u, dead};

    for (int c = blockIdx.x; c < a.ncols; c += gridDim.x)
        if (p2_column_ok(a, c, N, KREAL ? 1 : 2)) tc_column<P, N, KREAL>(A, c, st);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (t < 32)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(st.tbase), "r"(TP::TMEM_COLS));
}

}  // namespace lpk
