// PSF spectrum (step S0): K^ = DFT of the zero-padded PSF, Sec. 2.3 Eq. (10),
// computed once per (PSF, padded size) in FP64 and stored in FP32 in the
// column-major layout the column pass reads.
//
// The PSF is placed with its centre pixel at index (0,0) of the Ny x Nx
// padded grid (negative offsets wrap to the far end).  With that placement
// the circular convolution of Sec. 2.5 needs no crop offset for the
// same-size output, and the spectrum of a point-symmetric PSF is real.
//
// Pipeline (all on the caller's stream, FP64):
//   scatter rows of K into hk x Nx (wrap in x)  ->  FFT along x
//   scatter the first Nx/2+1 columns into Ny x (Nx/2+1) (wrap in y)  ->  FFT along y
//   scale by 1/(2 Ny Nx) and store transposed as FP32: real part only when
//   the PSF is point-symmetric (exact compare), complex otherwise.
// The FFT is a global-memory Stockham pass per radix (2, 3, 4, 5, 7, 8)
// with FP64 twiddles from sincospi; it is off the per-map hot path.
#include "fft_core.cuh"
#include "lp_internal.h"

namespace lpk {

template <int R, int DIR>
__global__ void fft64_stage(const double2* __restrict__ in, double2* __restrict__ out, int N,
                            int Ns, long long es, long long bs, int nb, int batch_fast)
{
    const long long NB = N / R;
    const long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= NB * nb) return;
    long long j, b;
    if (batch_fast) {
        b = g % nb;
        j = g / nb;
    } else {
        j = g % NB;
        b = g / NB;
    }
    double2 v[R];
#pragma unroll
    for (int m = 0; m < R; ++m) v[m] = in[b * bs + (j + m * NB) * es];
    const long long k = j % Ns;
    if (Ns > 1) {
        const long long n = (long long)Ns * R;
#pragma unroll
        for (int m = 1; m < R; ++m) {
            const long long tt = (k * m) % n;
            double s, c;
            sincospi(2.0 * (double)tt / (double)n, &s, &c);
            v[m] = cmul(v[m], mk<double2>(c, DIR * s));
        }
    }
    Dft<R, DIR, double2>::run(v);
    const long long base = (j / Ns) * Ns * R + k;
#pragma unroll
    for (int m = 0; m < R; ++m) out[b * bs + (base + m * Ns) * es] = v[m];
}

static int pick_radix64(int rem)
{
    if (rem % 8 == 0) return 8;
    if (rem % 4 == 0) return 4;
    if (rem % 2 == 0) return 2;
    if (rem % 3 == 0) return 3;
    if (rem % 5 == 0) return 5;
    if (rem % 7 == 0) return 7;
    return 0;
}

template <int DIR>
static cudaError_t launch_stage64(int R, const double2* in, double2* out, int N, int Ns,
                                  long long es, long long bs, int nb, int batch_fast,
                                  cudaStream_t st)
{
    const long long total = (long long)(N / R) * nb;
    const int thr = 256;
    const unsigned blocks = (unsigned)((total + thr - 1) / thr);
    switch (R) {
    case 2: fft64_stage<2, DIR><<<blocks, thr, 0, st>>>(in, out, N, Ns, es, bs, nb, batch_fast); break;
    case 3: fft64_stage<3, DIR><<<blocks, thr, 0, st>>>(in, out, N, Ns, es, bs, nb, batch_fast); break;
    case 4: fft64_stage<4, DIR><<<blocks, thr, 0, st>>>(in, out, N, Ns, es, bs, nb, batch_fast); break;
    case 5: fft64_stage<5, DIR><<<blocks, thr, 0, st>>>(in, out, N, Ns, es, bs, nb, batch_fast); break;
    case 7: fft64_stage<7, DIR><<<blocks, thr, 0, st>>>(in, out, N, Ns, es, bs, nb, batch_fast); break;
    case 8: fft64_stage<8, DIR><<<blocks, thr, 0, st>>>(in, out, N, Ns, es, bs, nb, batch_fast); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// Forward FFT of nb transforms of length N; element stride es, batch stride
// bs (elements).  Ping-pongs between a and tmp; *result gets the buffer that
// holds the output.
cudaError_t fft64_forward(double2* a, double2* tmp, int N, long long es, long long bs, int nb,
                          int batch_fast, cudaStream_t st, double2** result)
{
    double2* src = a;
    double2* dst = tmp;
    int Ns = 1, rem = N;
    while (rem > 1) {
        const int R = pick_radix64(rem);
        if (R == 0) return cudaErrorInvalidValue;
        cudaError_t e = launch_stage64<-1>(R, src, dst, N, Ns, es, bs, nb, batch_fast, st);
        if (e != cudaSuccess) return e;
        Ns *= R;
        rem /= R;
        double2* x = src;
        src = dst;
        dst = x;
    }
    *result = src;
    return cudaSuccess;
}

bool fft64_supported(int N)
{
    int rem = N;
    while (rem > 1) {
        const int R = pick_radix64(rem);
        if (R == 0) return false;
        rem /= R;
    }
    return N >= 1;
}

__global__ void psf_symmetry(const double* __restrict__ K, int hk, int wk, int* asym)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)hk * wk) return;
    const int y = (int)(i / wk), x = (int)(i % wk);
    if (K[i] != K[(long long)(hk - 1 - y) * wk + (wk - 1 - x)]) atomicOr(asym, 1);
}

__global__ void psf_scatter_rows(const double* __restrict__ K, int hk, int wk, int Nx, int cx,
                                 double2* __restrict__ W1)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)hk * wk) return;
    const int y = (int)(i / wk), x = (int)(i % wk);
    int xx = x - cx;
    if (xx < 0) xx += Nx;
    W1[(long long)y * Nx + xx] = mk<double2>(K[i], 0.0);
}

__global__ void psf_scatter_cols(const double2* __restrict__ W1, int hk, int Nx, int ncols,
                                 int Ny, int cy, double2* __restrict__ W2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)hk * ncols) return;
    const int y = (int)(i / ncols), c = (int)(i % ncols);
    int yy = y - cy;
    if (yy < 0) yy += Ny;
    W2[(long long)yy * ncols + c] = W1[(long long)y * Nx + c];
}

// dst[c][u] = scale * W2[u][c], 32 x 32 tiles through shared memory
__global__ void psf_store_spectrum(const double2* __restrict__ W2, int Ny, int ncols, double scale,
                                   int real_only, void* dst, long long ldK)
{
    __shared__ double2 tile[32][33];
    const int u0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int u = u0 + r, c = c0 + threadIdx.x;
        if (u < Ny && c < ncols) tile[r][threadIdx.x] = W2[(long long)u * ncols + c];
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int c = c0 + r, u = u0 + threadIdx.x;
        if (u < Ny && c < ncols) {
            const double2 z = tile[threadIdx.x][r];
            if (real_only)
                static_cast<float*>(dst)[(long long)c * ldK + u] = (float)(z.x * scale);
            else
                static_cast<float2*>(dst)[(long long)c * ldK + u] =
                    make_float2((float)(z.x * scale), (float)(z.y * scale));
        }
    }
}

// order-independent 64-bit fingerprint of the PSF values (cache key).  mix64
// is the SplitMix64 output finaliser (Steele, Lea and Flood, "Fast
// splittable pseudorandom number generators", OOPSLA 2014): its published
// shift and multiplier constants, applied to value bits and index.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void psf_fingerprint(const double* __restrict__ K, long long n, unsigned long long* out)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const unsigned long long bits = (unsigned long long)__double_as_longlong(K[i]);
    atomicAdd(out, mix64(bits ^ mix64((unsigned long long)i)));
}

cudaError_t psf_fingerprint_launch(const double* K, long long n, unsigned long long* d_out,
                                   cudaStream_t st)
{
    const unsigned blocks = (unsigned)((n + 255) / 256);
    psf_fingerprint<<<blocks, 256, 0, st>>>(K, n, d_out);
    return cudaGetLastError();
}

__global__ void psf_compare(const double* __restrict__ a, const double* __restrict__ b, long long n,
                            int* diff)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (__double_as_longlong(a[i]) != __double_as_longlong(b[i])) atomicOr(diff, 1);
}

cudaError_t psf_compare_launch(const double* a, const double* b, long long n, int* d_diff, cudaStream_t st)
{
    psf_compare<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n, d_diff);
    return cudaGetLastError();
}

cudaError_t psf_symmetry_launch(const double* K, int hk, int wk, int* d_asym, cudaStream_t st)
{
    const long long n = (long long)hk * wk;
    psf_symmetry<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(K, hk, wk, d_asym);
    return cudaGetLastError();
}

// Full spectrum build.  W1 holds hk*Nx, W2a/W2b each Ny*ncols complex128.
cudaError_t psf_spectrum_build(const double* K, int hk, int wk, int Ny, int Nx, int real_only,
                               void* dst, long long ldK, double2* W1, double2* W1b,
                               double2* W2a, double2* W2b, cudaStream_t st)
{
    const int ncols = Nx / 2 + 1;
    const int cy = (hk - 1) / 2, cx = (wk - 1) / 2;
    cudaError_t e;
    if ((e = cudaMemsetAsync(W1, 0, sizeof(double2) * (size_t)hk * Nx, st)) != cudaSuccess) return e;
    {
        const long long n = (long long)hk * wk;
        psf_scatter_rows<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(K, hk, wk, Nx, cx, W1);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    double2* rows = nullptr;
    if ((e = fft64_forward(W1, W1b, Nx, 1, Nx, hk, 0, st, &rows)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(W2a, 0, sizeof(double2) * (size_t)Ny * ncols, st)) != cudaSuccess) return e;
    {
        const long long n = (long long)hk * ncols;
        psf_scatter_cols<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(rows, hk, Nx, ncols, Ny, cy, W2a);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    double2* cols = nullptr;
    if ((e = fft64_forward(W2a, W2b, Ny, ncols, 1, ncols, 1, st, &cols)) != cudaSuccess) return e;
    const double scale = 1.0 / (2.0 * (double)Ny * (double)Nx);
    dim3 grid((ncols + 31) / 32, (Ny + 31) / 32), block(32, 8);
    psf_store_spectrum<<<grid, block, 0, st>>>(cols, Ny, ncols, scale, real_only, dst, ldK);
    return cudaGetLastError();
}

}  // namespace lpk
