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

struct P1Args;
struct P2Args;
struct P3Args;
struct P2MArgs;
struct P2TcArgs;

// One supported FFT length with its compiled FP32 kernels.
struct SizeKernels {
    int N;
    int nstages;
    int radices[6];      // forward order
    int threads;         // threads per transform
    int f1, f3;          // transforms per block in the row passes
    int smem_bytes;      // dynamic shared memory of one transform
    int batch;           // several spectra: one forward column transform, parked
    cudaError_t (*set_attrs)();
    // launchers: pick the persistent prefetching kernel when its shared
    // memory fits, the one-unit-per-block kernel otherwise
    cudaError_t (*p1)(const P1Args&, cudaStream_t);
    cudaError_t (*p2)(const P2Args&, bool kreal, cudaStream_t);
    cudaError_t (*p2m)(const P2MArgs&, bool kreal, cudaStream_t);
    cudaError_t (*p3)(const P3Args&, int nspec, cudaStream_t);
    // split-precision (BF16 hi/lo) tensor-core column pass, one spectrum per
    // launch; tc_smem = 0 where this length has none
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
cudaError_t psf_spectrum_build(const double* K, int hk, int wk, int Ny, int Nx, int real_only,
                               void* dst, long long ldK, double2* W1, double2* W1b,
                               double2* W2a, double2* W2b, cudaStream_t st);

}  // namespace lpk
