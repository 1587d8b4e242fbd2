// The three FP32 passes of the Fourier-domain convolution (Sec. 2.3 Eq. (9),
// workflow of Sec. 2.5 / Fig. 1): zero padding is implicit, the spectrum
// product sits between the forward and inverse column transforms, and the
// crop is a predicate on the last stores.
//
//   P1  rows:    two real rows a, b packed as z = a + i b, length-Nx forward
//                FFT, split into the half spectra of a and b (Hermitian
//                symmetry), stored transposed: T[c][i], c in [0, Nx/2].
//   P2  columns: per column c, length-Ny forward FFT of T[c][0..H) (rows
//                >= H are the zero padding), multiply by the PSF spectrum
//                K^[c][.] (pre-scaled by 1/(2 Ny Nx)), inverse FFT, keep the
//                output rows of the crop window.  With n spectra the forward
//                result stays in registers and is reused n times.
//   P3  rows:    Hermitian extension of two rows' half spectra packed as
//                Z = A + i B, length-Nx inverse FFT, real part -> row a,
//                imaginary part -> row b, keep the crop columns.
//
// Layouts (element = complex64 unless stated):
//   L    FP32, row-major H x W, leading dimension ldl (elements)
//   T    (Nx/2+1) rows of ldT >= 2 ceil(H/2) elements
//   K^   (Nx/2+1) rows of ldK elements: FP32 (point-symmetric PSF, real
//        spectrum) or complex64
//   U    per spectrum (Nx/2+1) rows of ldU >= 2 ceil(Hout/2) elements
//   out  FP32 row-major Hout x Wout, leading dimension ldo
#pragma once

#include "fft_core.cuh"

namespace lpk {

constexpr int kMaxSpectraPerLaunch = 32;

struct P1Args {
    const float* L;
    long long ldl;
    int H, W;
    float2* T;
    long long ldT;
    int npairs;  // ceil(H/2)
    int ncols;   // Nx/2 + 1
    TwChain tw;  // forward chain of the row plan
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
};

struct P3Args {
    const float2* U;
    long long ldU;
    long long specU;
    int Hout, npairs;
    float* out[kMaxSpectraPerLaunch];
    long long ldo;
    int c0;  // first kept column (mod Nx)
    int Wout;
    int ncols;
    TwChain tw;  // reversed chain of the row plan
};

template <int N, class FwdSeq>
struct Plan {
    using Fwd = FwdSeq;
    using Inv = Reverse<FwdSeq>;
    static_assert(SeqInfo<Fwd>::product == N, "radices must multiply to N");
    static constexpr int R0 = SeqInfo<Fwd>::first;   // first forward radix
    static constexpr int RL = SeqInfo<Fwd>::last;    // last forward radix
    static constexpr int T = ((N / SeqInfo<Fwd>::min_r) + 31) / 32 * 32;  // threads per FFT
    // shared memory (complex elements) of one transform: the larger padded
    // extent of the forward and the reversed chain
    static constexpr int SMEM_ELEMS = ChainExtent<Fwd>::value > ChainExtent<Inv>::value
                                          ? ChainExtent<Fwd>::value
                                          : ChainExtent<Inv>::value;
    static constexpr int SMEM_BYTES = 8 * SMEM_ELEMS;
    static_assert(T <= 1024, "too many threads per transform");
};

// ---------------------------------------------------------------------------
// P1: row R2C of two packed rows per transform, F transforms per block.
// ---------------------------------------------------------------------------
template <class P, int N, int F>
__global__ void __launch_bounds__(P::T * F) p1_rows(const P1Args a)
{
    extern __shared__ float2 smem2[];
    constexpr int T = P::T;
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int RL = P::RL, NBL = N / RL;
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    float2* sm = smem2 + f * P::SMEM_ELEMS;
    const int pair = blockIdx.x * F + f;
    const int ra = 2 * pair, rb = ra + 1;
    const bool va = ra < a.H, vb = rb < a.H;
    const float* La = a.L + (long long)ra * a.ldl;
    const float* Lb = a.L + (long long)rb * a.ldl;

    float2 v[R0];
    if (t < NB0) {
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int col = t + m * NB0;
            const bool in = col < a.W;
            v[m].x = (in && va) ? __ldg(La + col) : 0.f;
            v[m].y = (in && vb) ? __ldg(Lb + col) : 0.f;
        }
    }
    using FwdChain = Chain<N, -1, 1, 0, typename P::Fwd>;
    FwdChain::run(v, t, sm, a.tw, [&](float2(&z)[RL], int j, bool act) {
        __syncthreads();
        if (act) {
#pragma unroll
            for (int m = 0; m < RL; ++m) sm[j + m * NBL] = z[m];
        }
        __syncthreads();
        if (pair < a.npairs) {
            float4* Tq = reinterpret_cast<float4*>(a.T);
            for (int c = t; c < a.ncols; c += T) {
                const int cm = (c == 0) ? 0 : N - c;
                const float2 zc = sm[c], zm = sm[cm];
                const float zr = zc.x, zi = zc.y;
                const float wr = zm.x, wi = -zm.y;
                // 2 X_a = Z[c] + conj Z[N-c] ; 2 X_b = -i (Z[c] - conj Z[N-c])
                float4 o;
                o.x = zr + wr;
                o.y = zi + wi;
                o.z = zi - wi;
                o.w = -(zr - wr);
                Tq[((long long)c * a.ldT) / 2 + pair] = o;
            }
        }
    });
}

// ---------------------------------------------------------------------------
// P2: per column forward FFT, spectrum product, inverse FFT, row crop.
// ---------------------------------------------------------------------------
template <class P, int N, bool KREAL, bool MULTI>
__global__ void __launch_bounds__(P::T) p2_cols(const P2Args a)
{
    extern __shared__ float2 smem2[];
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int RL = P::RL, NBL = N / RL;
    float2* sm = smem2;
    const int c = blockIdx.x;
    const int t = threadIdx.x;
    const float2* col = a.T + (long long)c * a.ldT;

    float2 v[R0];
    if (t < NB0) {
#pragma unroll
        for (int m = 0; m < R0; ++m) {
            const int row = t + m * NB0;
            v[m] = row < a.H ? __ldg(col + row) : make_float2(0.f, 0.f);
        }
    }
    using FwdChain = Chain<N, -1, 1, 0, typename P::Fwd>;
    using InvChain = Chain<N, +1, 1, 0, typename P::Inv>;
    auto product = [&](float2* g, const float2* fz, int s, int j) {
        if constexpr (KREAL) {
            const float* kc = static_cast<const float*>(a.K[s]) + (long long)c * a.ldK + j;
#pragma unroll
            for (int m = 0; m < RL; ++m) {
                const float k = __ldg(kc + m * NBL);
                g[m] = make_float2(fz[m].x * k, fz[m].y * k);
            }
        } else {
            const float2* kc = static_cast<const float2*>(a.K[s]) + (long long)c * a.ldK + j;
#pragma unroll
            for (int m = 0; m < RL; ++m) g[m] = cmul(fz[m], __ldg(kc + m * NBL));
        }
    };
    auto inverse = [&](float2(&g)[RL], int s, int j) {
        float2* Uc = a.U + (long long)s * a.specU + (long long)c * a.ldU;
        InvChain::run(g, j, sm, a.twi, [&](float2(&o)[R0], int j2, bool act2) {
            if (act2) {
#pragma unroll
                for (int m = 0; m < R0; ++m) {
                    int rr = j2 + m * NB0 - a.r0;
                    if (rr < 0) rr += N;
                    if (rr < a.Hout) Uc[rr] = o[m];
                }
            }
            if (a.HoutPad != a.Hout && j2 == 0) Uc[a.Hout] = make_float2(0.f, 0.f);
        });
    };
    FwdChain::run(v, t, sm, a.twf, [&](float2(&fz)[RL], int j, bool act) {
        if constexpr (MULTI) {
#pragma unroll 1
            for (int s = 0; s < a.nspec; ++s) {
                float2 g[RL];
                if (act) product(g, fz, s, j);
                inverse(g, s, j);
            }
        } else {
            if (act) product(fz, fz, 0, j);
            inverse(fz, 0, j);
        }
    });
}

// ---------------------------------------------------------------------------
// P3: row C2R of two packed rows per transform, F transforms per block,
// blockIdx.y selects the spectrum.
// ---------------------------------------------------------------------------
template <class P, int N, int F>
__global__ void __launch_bounds__(P::T * F) p3_rows(const P3Args a)
{
    extern __shared__ float2 smem2[];
    constexpr int T = P::T;
    constexpr int RI = SeqInfo<typename P::Inv>::first, NBI = N / RI;
    constexpr int RJ = SeqInfo<typename P::Inv>::last, NBJ = N / RJ;
    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    float2* sm = smem2 + f * P::SMEM_ELEMS;
    const int pair = blockIdx.x * F + f;
    const int sidx = blockIdx.y;
    const int ra = 2 * pair, rb = ra + 1;
    const float4* Uq = reinterpret_cast<const float4*>(a.U + (long long)sidx * a.specU);
    const long long ldq = a.ldU / 2;
    const bool live = pair < a.npairs;
    const bool vb = rb < a.Hout;

    float2 v[RI];
    if (t < NBI) {
#pragma unroll
        for (int m = 0; m < RI; ++m) {
            const int k = t + m * NBI;
            float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
            const bool lo = k < a.ncols;
            if (live) q = __ldg(Uq + (long long)(lo ? k : N - k) * ldq + pair);
            if (!vb) {
                q.z = 0.f;
                q.w = 0.f;
            }
            // Z[k] = A[k] + i B[k]; for k > Nx/2, A[k] = conj A[N-k], same for B
            v[m] = lo ? make_float2(q.x - q.w, q.y + q.z) : make_float2(q.x + q.w, q.z - q.y);
        }
    }
    using InvChain = Chain<N, +1, 1, 0, typename P::Inv>;
    InvChain::run(v, t, sm, a.tw, [&](float2(&o)[RJ], int j, bool act) {
        if (act && live) {
            float* oa = a.out[sidx] + (long long)ra * a.ldo;
            float* ob = oa + a.ldo;
#pragma unroll
            for (int m = 0; m < RJ; ++m) {
                int cc = j + m * NBJ - a.c0;
                if (cc < 0) cc += N;
                if (cc < a.Wout) {
                    oa[cc] = o[m].x;
                    if (vb) ob[cc] = o[m].y;
                }
            }
        }
    });
}


// ---------------------------------------------------------------------------
// P2 for Sec. 2.2 Eq. (4): several source classes, one PSF each.  The
// forward column transform of each class's T is multiplied by its spectrum
// and accumulated in registers; one inverse transform follows.
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
};

template <class P, int N, bool KREAL>
__global__ void __launch_bounds__(P::T) p2_multiclass(const P2MArgs a)
{
    extern __shared__ float2 smem2[];
    constexpr int R0 = P::R0, NB0 = N / R0;
    constexpr int RL = P::RL, NBL = N / RL;
    float2* sm = smem2;
    const int c = blockIdx.x;
    const int t = threadIdx.x;
    using FwdChain = Chain<N, -1, 1, 0, typename P::Fwd>;
    using InvChain = Chain<N, +1, 1, 0, typename P::Inv>;

    float2 acc[RL];
#pragma unroll
    for (int m = 0; m < RL; ++m) acc[m] = make_float2(0.f, 0.f);
#pragma unroll 1
    for (int q = 0; q < a.nclass; ++q) {
        const float2* col = a.T[q] + (long long)c * a.ldT;
        float2 v[R0];
        if (t < NB0) {
#pragma unroll
            for (int m = 0; m < R0; ++m) {
                const int row = t + m * NB0;
                v[m] = row < a.H ? __ldg(col + row) : make_float2(0.f, 0.f);
            }
        }
        FwdChain::run(v, t, sm, a.twf, [&](float2(&fz)[RL], int j, bool act) {
            if (act) {
                if constexpr (KREAL) {
                    const float* kc = static_cast<const float*>(a.K[q]) + (long long)c * a.ldK;
#pragma unroll
                    for (int m = 0; m < RL; ++m) {
                        const float k = __ldg(kc + j + m * NBL);
                        acc[m].x += fz[m].x * k;
                        acc[m].y += fz[m].y * k;
                    }
                } else {
                    const float2* kc = static_cast<const float2*>(a.K[q]) + (long long)c * a.ldK;
#pragma unroll
                    for (int m = 0; m < RL; ++m) acc[m] = cadd(acc[m], cmul(fz[m], __ldg(kc + j + m * NBL)));
                }
            }
        });
        __syncthreads();  // the next class's forward reuses re/im
    }
    float2* Uc = a.U + (long long)c * a.ldU;
    InvChain::run(acc, t, sm, a.twi, [&](float2(&o)[R0], int j2, bool act2) {
        if (act2) {
#pragma unroll
            for (int m = 0; m < R0; ++m) {
                int rr = j2 + m * NB0 - a.r0;
                if (rr < 0) rr += N;
                if (rr < a.Hout) Uc[rr] = o[m];
            }
        }
        if (a.HoutPad != a.Hout && j2 == 0) Uc[a.Hout] = make_float2(0.f, 0.f);
    });
}

}  // namespace lpk
