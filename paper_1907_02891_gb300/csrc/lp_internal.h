// Internal interfaces between the C-ABI layer (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lpk {

// Per-stage twiddle tables of one Stockham chain: table s (s >= 1) holds
// exp(-i 2 pi k m / (Ns R_s)) at [(m-1) Ns + k], k < Ns, 1 <= m < R_s,
// with Ns = R_0 ... R_{s-1}.
struct TwChain {
    const float2* p[6];
};

struct P2Args;
struct P2TcArgs;
struct P1v2Args;
struct P2v2Args;
struct P3v2Args;
struct P2Mv2Args;

// Tables of the in-place engine (fft2.cuh) for one length N: the twiddles
// W[i] = exp(-i 2 pi i / N), i < N, as {cos, sin}, and the position of every
// frequency after the forward transform.
struct TwTab2 {
    const float2* w;
    const unsigned short* pos;
};

// One supported FFT length with its compiled kernels.
struct SizeKernels {
    int N;
    // FP32 passes on the in-place engine
    int nstages;
    int radices[8];   // forward (DIF) order
    int pair[3];      // two transforms per block in P1, P2, P3
    int threads[3];
    int batch;        // several spectra: one forward column transform for all
    cudaError_t (*set_attrs)();
    cudaError_t (*p1)(const P1v2Args&, cudaStream_t);
    cudaError_t (*p2)(const P2v2Args&, bool kreal, cudaStream_t);
    cudaError_t (*p2m)(const P2Mv2Args&, bool kreal, cudaStream_t);
    cudaError_t (*p3)(const P3v2Args&, int nspec, cudaStream_t);
    // split-precision (BF16 hi/lo) tensor-core column pass, one spectrum per
    // launch, on its own Stockham radix plan; tc_smem = 0 where this length
    // has none
    int tc_nstages;
    int tc_radices[6];
    int tc_threads;
    int tc_smem;
    cudaError_t (*p2tc)(const P2TcArgs&, bool kreal, cudaStream_t);
};

// generated registry (one translation unit per size)
extern const SizeKernels* const kAllSizes[];
extern const int kNumSizes;

// FP64 spectrum pipeline (spectrum.cu)
bool fft64_supported(int N);
cudaError_t psf_fingerprint_launch(const double* K, long long n, unsigned long long* d_out,
                                   cudaStream_t st);
cudaError_t psf_symmetry_launch(const double* K, int hk, int wk, int* d_asym, cudaStream_t st);
// *d_diff |= 1 where a[i] and b[i] differ in any bit (i < n)
cudaError_t psf_compare_launch(const double* a, const double* b, long long n, int* d_diff, cudaStream_t st);
// pos = NULL: natural layout (rows c of ldK frequencies; the tensor-core
// pass); else the FP32 column pass's layout (column pairs, position order)
cudaError_t psf_spectrum_build(const double* K, int hk, int wk, int Ny, int Nx, int real_only,
                               void* dst, long long ldK, double2* W1, double2* W1b,
                               double2* W2a, double2* W2b, const unsigned short* pos, cudaStream_t st);
cudaError_t psf_copy_natural_launch(const void* src, int ny, int ncols, long long ldK, int real_only,
                                    const unsigned short* pos, float* dst, cudaStream_t st);

}  // namespace lpk
