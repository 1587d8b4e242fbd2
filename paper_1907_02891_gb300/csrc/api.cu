// C-ABI layer of liblp.so: argument validation, contexts, FFT plans and
// twiddle tables, the device-resident PSF-spectrum cache, per-stream
// workspaces and the launch sequence of the map (include/lp.h documents
// every entry point).
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <algorithm>
#include <vector>

#include "../../include/lp.h"
#include "conv_kernels.cuh"
#include "lp_internal.h"
#include "tc_kernels.cuh"
#include "lp_runtime.h"

using namespace lpk;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

lp_status lp_fail(lp_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CUDA_TRY(call)                                                                     \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return lp_fail(e_ == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,     \
                           "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__,      \
                           __LINE__);                                                      \
    } while (0)

extern "C" const char* lp_last_error(void) { return g_err.c_str(); }
extern "C" int lp_version(void) { return 100; }

// ---------------------------------------------------------------------------
// supported sizes
// ---------------------------------------------------------------------------
static const SizeKernels* find_size(int n)
{
    for (int i = 0; i < kNumSizes; ++i)
        if (kAllSizes[i]->N == n) return kAllSizes[i];
    return nullptr;
}

extern "C" int lp_num_supported_sizes(void) { return kNumSizes; }
extern "C" int lp_supported_size_at(int i) { return (i >= 0 && i < kNumSizes) ? kAllSizes[i]->N : -1; }
extern "C" int lp_supported_size(int n)
{
    int best = -1;
    for (int i = 0; i < kNumSizes; ++i) {
        const int N = kAllSizes[i]->N;
        if (N >= n && (best < 0 || N < best)) best = N;
    }
    return best;
}

extern "C" int lp_split_supported(int n)
{
    const SizeKernels* k = find_size(n);
    return (k && k->tc_smem > 0) ? 1 : 0;
}

// smallest length >= n that has the split-precision tensor-core column pass
static int tc_supported_size(int n)
{
    int best = -1;
    for (int i = 0; i < kNumSizes; ++i) {
        const int N = kAllSizes[i]->N;
        if (N >= n && kAllSizes[i]->tc_smem > 0 && (best < 0 || N < best)) best = N;
    }
    return best;
}

// Padded length of one dimension for the tiled map: the supported length
// N >= k that minimises the transformed points of that dimension, tiles * N
// with one tile where n <= N - (k - 1) / 2, else ceil(n / (N - k + 1))
// (ties: fewer tiles); with tc, only lengths that have the tensor-core
// column pass.
static int tile_length(int n, int k, bool tc)
{
    long long best_cost = -1;
    int best = -1, best_tiles = 0;
    const int c = (k - 1) / 2;
    for (int i = 0; i < kNumSizes; ++i) {
        const int N = kAllSizes[i]->N;
        if (N < k || (tc && kAllSizes[i]->tc_smem == 0)) continue;
        const int t = N - k + 1;
        const int tiles = n <= N - c ? 1 : (n + t - 1) / t;   // as lp_map_tiled cuts them
        const long long cost = (long long)tiles * N;
        if (best < 0 || cost < best_cost || (cost == best_cost && tiles < best_tiles)) {
            best = N;
            best_cost = cost;
            best_tiles = tiles;
        }
    }
    return best;
}

extern "C" lp_status lp_tiled_pad(int h, int w, int hk, int wk, lp_precision prec, int* pad_ny, int* pad_nx)
{
    if (!pad_ny || !pad_nx) return lp_fail(LP_ERR_INVALID, "lp_tiled_pad: NULL argument");
    *pad_ny = *pad_nx = -1;
    if (h < 1 || w < 1) return lp_fail(LP_ERR_INVALID, "lp_tiled_pad: empty map %d x %d", h, w);
    if (hk < 1 || wk < 1 || hk % 2 == 0 || wk % 2 == 0)
        return lp_fail(LP_ERR_INVALID, "lp_tiled_pad: PSF sides must be odd and >= 1 (got %d x %d)", hk, wk);
    if (prec != LP_PREC_FP32 && prec != LP_PREC_SPLIT_BF16)
        return lp_fail(LP_ERR_UNSUPPORTED, "lp_tiled_pad: precision %d is not built", (int)prec);
    const int ny = tile_length(h, hk, prec == LP_PREC_SPLIT_BF16), nx = tile_length(w, wk, false);
    if (ny < 0 || nx < 0) return lp_fail(LP_ERR_UNSUPPORTED, "lp_tiled_pad: no supported length holds the PSF");
    *pad_ny = ny;
    *pad_nx = nx;
    return LP_OK;
}

// ---------------------------------------------------------------------------
// device guard
// ---------------------------------------------------------------------------
namespace {
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};
}  // namespace

static void free_spectrum(lp_ctx* ctx, lp_spectrum* s);

// ---------------------------------------------------------------------------
// context internals
// ---------------------------------------------------------------------------
lp_status lp_ctx_alloc(lp_ctx* ctx, size_t bytes, void** p)
{
    *p = nullptr;
    if (bytes == 0) return LP_OK;
    {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        if (ctx->budget && ctx->used + bytes > ctx->budget)
            return lp_fail(LP_ERR_OOM, "HBM budget: %zu bytes held + %zu requested > %zu", ctx->used,
                           bytes, ctx->budget);
        ctx->used += bytes;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        std::lock_guard<std::mutex> g(ctx->mem_mu);
        ctx->used -= bytes;
        *p = nullptr;
        return lp_fail(e == cudaErrorMemoryAllocation ? LP_ERR_OOM : LP_ERR_CUDA,
                       "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    return LP_OK;
}

void lp_ctx_free(lp_ctx* ctx, void* p, size_t bytes)
{
    if (!p) return;
    cudaFree(p);
    std::lock_guard<std::mutex> g(ctx->mem_mu);
    ctx->used -= bytes;
}

// twiddle tables of one chain: stage s >= 1 holds (R_s - 1) * Ns entries
static size_t chain_table_entries(const int* r, int ns)
{
    size_t tot = 0;
    long Ns = r[0];
    for (int s = 1; s < ns; ++s) {
        tot += (size_t)(r[s] - 1) * Ns;
        Ns *= r[s];
    }
    return tot;
}

static void fill_chain_tables(const int* r, int ns, std::vector<float2>& host, size_t base,
                              size_t* offs)
{
    long Ns = r[0];
    size_t o = base;
    offs[0] = o;
    for (int s = 1; s < ns; ++s) {
        offs[s] = o;
        const long n = Ns * r[s];
        for (int m = 1; m < r[s]; ++m)
            for (long k = 0; k < Ns; ++k) {
                const long t = (k * m) % n;
                const double th = 2.0 * M_PI * (double)t / (double)n;
                host[o + (size_t)(m - 1) * Ns + k] = make_float2((float)std::cos(th), (float)-std::sin(th));
            }
        o += (size_t)(r[s] - 1) * Ns;
        Ns *= r[s];
    }
}

// BF16 of x, round to nearest even (finite inputs)
static uint16_t bf16_rn(float x)
{
    uint32_t u;
    std::memcpy(&u, &x, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}

static float bf16_to_float(uint16_t h)
{
    const uint32_t u = (uint32_t)h << 16;
    float x;
    std::memcpy(&x, &u, 4);
    return x;
}

// bytes of the split-BF16 DFT matrices of one chain (hi + lo per stage)
static size_t tc_chain_bytes(const int* r, int ns)
{
    size_t b = 0;
    for (int s = 0; s < ns; ++s) b += 2ull * ru16(2 * r[s]) * ru16(2 * r[s]) * 2;
    return b;
}

// The split-BF16 DFT matrices of a chain for the tensor-core column pass.
// Stage s (radix R, Kp = 16 ceil(2R / 16)) maps a butterfly's inputs x_q
// (Re, Im interleaved: columns 2q, 2q+1) to its outputs y_k (rows 2k, 2k+1),
// y_k = sum_q x_q exp(dir i 2 pi k q / R) (Eq. (10) of radix R), as the
// real Kp x Kp matrix with blocks [c -s; s c], c + i s = exp(dir i 2 pi kq/R),
// zero elsewhere.  Each matrix is stored as hi = bf16(M) then
// lo = bf16(M - hi), element (n, k) at ((n / 8) (Kp / 8) + k / 8) 64 +
// (n mod 8) 8 + k mod 8 (8 x 8 core matrices, K-major).
static void fill_tc_mats(const int* r, int ns, int dir, uint16_t* dst)
{
    for (int s = 0; s < ns; ++s) {
        const int R = r[s], KP = ru16(2 * R), KG = KP / 8;
        std::vector<double> M((size_t)KP * KP, 0.0);
        for (int k = 0; k < R; ++k)
            for (int q = 0; q < R; ++q) {
                const double th = 2.0 * M_PI * (double)((k * q) % R) / (double)R;
                const double c = std::cos(th), sn = dir * std::sin(th);
                M[(size_t)(2 * k) * KP + 2 * q] = c;
                M[(size_t)(2 * k) * KP + 2 * q + 1] = -sn;
                M[(size_t)(2 * k + 1) * KP + 2 * q] = sn;
                M[(size_t)(2 * k + 1) * KP + 2 * q + 1] = c;
            }
        uint16_t* hi = dst;
        uint16_t* lo = dst + (size_t)KP * KP;
        for (int n = 0; n < KP; ++n)
            for (int k = 0; k < KP; ++k) {
                const double v = M[(size_t)n * KP + k];
                const uint16_t h = bf16_rn((float)v);
                const uint16_t l = bf16_rn((float)(v - (double)bf16_to_float(h)));
                const size_t off = ((size_t)(n / 8) * KG + k / 8) * 64 + (n % 8) * 8 + (k % 8);
                hi[off] = h;
                lo[off] = l;
            }
        dst += 2ull * KP * KP;
    }
}

// bytes of the twiddle step factors of one chain (stages s >= 1)
static size_t tc_step_bytes(const int* r, int ns)
{
    size_t b = 0;
    for (int s = 1; s < ns; ++s) b += (size_t)r[s - 1] * r[s] * sizeof(float2);
    return b;
}

// Step factors of the tensor-core column pass: the next stage's twiddle of
// output k of a butterfly with slot m is w0 * exp(dir i 2 pi m k / (R_{s-1} R_s)),
// stored at [m R_{s-1} + k] per stage s >= 1.
static void fill_tc_steps(const int* r, int ns, int dir, float2* dst)
{
    for (int s = 1; s < ns; ++s) {
        const int Rp = r[s - 1], R = r[s], n = Rp * R;
        for (int m = 0; m < R; ++m)
            for (int k = 0; k < Rp; ++k) {
                const double th = 2.0 * M_PI * (double)((m * k) % n) / (double)n;
                dst[m * Rp + k] = make_float2((float)std::cos(th), (float)(dir * std::sin(th)));
            }
        dst += (size_t)Rp * R;
    }
}

lp_status lp_get_plan(lp_ctx* ctx, int N, const PlanRec** out)
{
    std::lock_guard<std::mutex> g(ctx->plan_mu);
    auto it = ctx->plans.find(N);
    if (it != ctx->plans.end()) {
        *out = it->second.get();
        return LP_OK;
    }
    const SizeKernels* k = find_size(N);
    if (!k) return lp_fail(LP_ERR_UNSUPPORTED, "FFT length %d is not built into this library", N);
    int fwd[6], rev[6];
    const int ns = k->nstages;
    for (int s = 0; s < ns; ++s) {
        fwd[s] = k->radices[s];
        rev[s] = k->radices[ns - 1 - s];
    }
    const size_t nf = chain_table_entries(fwd, ns), nr = chain_table_entries(rev, ns);
    // one device block: twiddle tables, then (256-byte aligned) the split
    // DFT matrices of the tensor-core column pass where this length has one
    const size_t tw_bytes = (nf + nr + 1) * sizeof(float2);
    const size_t tc_off = (tw_bytes + 255) / 256 * 256;
    // (matrices of the forward stages -- the inverse chain runs in the
    // conjugate domain on the same ones --, then the step factors of the
    // forward and of the reversed chain, both with the forward sign)
    const size_t tcf = k->tc_smem > 0 ? tc_chain_bytes(fwd, ns) : 0;
    const size_t tsf = k->tc_smem > 0 ? tc_step_bytes(fwd, ns) : 0;
    const size_t tsr = k->tc_smem > 0 ? tc_step_bytes(rev, ns) : 0;
    const size_t total = k->tc_smem > 0 ? tc_off + (tcf + tsf + tsr + 15) / 16 * 16 : tw_bytes;
    std::vector<unsigned char> host(total, 0);
    float2* htw = reinterpret_cast<float2*>(host.data());
    std::vector<float2> tw(nf + nr + 1);
    size_t of[6] = {0}, orv[6] = {0};
    fill_chain_tables(fwd, ns, tw, 0, of);
    fill_chain_tables(rev, ns, tw, nf, orv);
    std::memcpy(htw, tw.data(), tw.size() * sizeof(float2));
    if (k->tc_smem > 0) {
        fill_tc_mats(fwd, ns, -1, reinterpret_cast<uint16_t*>(host.data() + tc_off));
        fill_tc_steps(fwd, ns, -1, reinterpret_cast<float2*>(host.data() + tc_off + tcf));
        fill_tc_steps(rev, ns, -1, reinterpret_cast<float2*>(host.data() + tc_off + tcf + tsf));
    }
    auto rec = std::make_unique<PlanRec>();
    rec->k = k;
    rec->bytes = total;
    void* d = nullptr;
    lp_status st = lp_ctx_alloc(ctx, rec->bytes, &d);
    if (st != LP_OK) return st;
    rec->tw = static_cast<float2*>(d);
    cudaError_t e = cudaMemcpy(d, host.data(), rec->bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lp_ctx_free(ctx, d, rec->bytes);
        return lp_fail(LP_ERR_CUDA, "twiddle upload: %s", cudaGetErrorString(e));
    }
    for (int s = 0; s < 6; ++s) {
        rec->fwd.p[s] = s < ns ? rec->tw + of[s] : nullptr;
        rec->rev.p[s] = s < ns ? rec->tw + orv[s] : nullptr;
    }
    if (k->tc_smem > 0) rec->tc_tables = static_cast<char*>(d) + tc_off;
    *out = rec.get();
    ctx->plans.emplace(N, std::move(rec));
    return LP_OK;
}

// per-stream workspace; grows (with a device sync) when a call needs more
bool lp_stream_capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return cs != cudaStreamCaptureStatusNone;
}

lp_status lp_get_workspace(lp_ctx* ctx, cudaStream_t s, size_t bytes, void** out)
{
    std::lock_guard<std::mutex> g(ctx->ws_mu);
    Workspace* w = nullptr;
    for (auto& x : ctx->ws)
        if (x.stream == s) w = &x;
    if (!w) {
        ctx->ws.push_back(Workspace{s, nullptr, 0});
        w = &ctx->ws.back();
    }
    if (w->bytes < bytes) {
        // growing synchronises the stream and allocates: neither may happen
        // inside a stream capture
        if (lp_stream_capturing(s))
            return lp_fail(LP_ERR_INVALID,
                           "workspace of %zu bytes needed while the stream is being captured (%zu held): "
                           "run the same call once before capturing, or use lp_map_noalloc",
                           bytes, w->bytes);
        if (w->ptr) {
            cudaStreamSynchronize(s);
            lp_ctx_free(ctx, w->ptr, w->bytes);
            w->ptr = nullptr;
            w->bytes = 0;
        }
        void* p = nullptr;
        lp_status st = lp_ctx_alloc(ctx, bytes, &p);
        if (st != LP_OK) return st;
        w->ptr = p;
        w->bytes = bytes;
    }
    *out = w->ptr;
    return LP_OK;
}

// ---------------------------------------------------------------------------
// create / destroy
// ---------------------------------------------------------------------------
extern "C" lp_status lp_create(lp_ctx** ctx, int device, size_t hbm_budget_bytes)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_create: ctx is NULL");
    *ctx = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return lp_fail(LP_ERR_CUDA, "lp_create: no CUDA device available");
    if (device < 0 || device >= ndev)
        return lp_fail(LP_ERR_INVALID, "lp_create: device %d out of range [0,%d)", device, ndev);
    DeviceGuard dg(device);
    if (!dg.ok) return lp_fail(LP_ERR_CUDA, "lp_create: cudaSetDevice(%d) failed", device);
    for (int i = 0; i < kNumSizes; ++i) CUDA_TRY(kAllSizes[i]->set_attrs());
    auto c = new (std::nothrow) lp_ctx();
    if (!c) return lp_fail(LP_ERR_OOM, "lp_create: host allocation failed");
    c->device = device;
    c->budget = hbm_budget_bytes;
    void* e = nullptr;
    lp_status st = lp_ctx_alloc(c, 64, &e);
    if (st != LP_OK) {
        delete c;
        return st;
    }
    c->d_err = static_cast<int*>(e);
    cudaMemset(c->d_err, 0, 64);
    *ctx = c;
    return LP_OK;
}

extern "C" void lp_destroy(lp_ctx* ctx)
{
    if (!ctx) return;
    DeviceGuard dg(ctx->device);
    lp_serve_shutdown(ctx);
    cudaDeviceSynchronize();
    for (auto& kv : ctx->spectra) free_spectrum(ctx, kv.second);
    ctx->spectra.clear();
    for (lp_spectrum* sp : ctx->released) free_spectrum(ctx, sp);
    ctx->released.clear();
    for (auto& w : ctx->ws) lp_ctx_free(ctx, w.ptr, w.bytes);
    ctx->ws.clear();
    for (auto& kv : ctx->plans) lp_ctx_free(ctx, kv.second->tw, kv.second->bytes);
    ctx->plans.clear();
    lp_ctx_free(ctx, ctx->staging, ctx->staging_bytes);
    lp_ctx_free(ctx, ctx->d_err, 64);
    for (auto& pe : ctx->tim_pending) {
        cudaEventDestroy(pe.start);
        cudaEventDestroy(pe.stop);
    }
    for (auto ev : ctx->tim_pool) cudaEventDestroy(ev);
    for (auto ev : ctx->hs_events) cudaEventDestroy(ev);
    for (auto ev : ctx->hs_lfree)
        if (ev) cudaEventDestroy(ev);
    for (auto ev : ctx->hs_ofree)
        if (ev) cudaEventDestroy(ev);
    if (ctx->hs_in) cudaStreamDestroy(ctx->hs_in);
    if (ctx->hs_out) cudaStreamDestroy(ctx->hs_out);
    if (ctx->hs_comp) cudaStreamDestroy(ctx->hs_comp);
    delete ctx;
}

extern "C" size_t lp_bytes_in_use(const lp_ctx* ctx)
{
    if (!ctx) return 0;
    std::lock_guard<std::mutex> g(const_cast<lp_ctx*>(ctx)->mem_mu);
    return ctx->used;
}

// ---------------------------------------------------------------------------
// spectra
// ---------------------------------------------------------------------------
extern "C" lp_status lp_kernel_spectrum(lp_ctx* ctx, const double* K, int hk, int wk, int max_h,
                                        int max_w, int pad_ny, int pad_nx, lp_precision prec,
                                        void* stream, lp_spectrum** out)
{
    if (out) *out = nullptr;
    if (!ctx || !K || !out) return lp_fail(LP_ERR_INVALID, "lp_kernel_spectrum: NULL argument");
    if (hk < 1 || wk < 1 || hk % 2 == 0 || wk % 2 == 0)
        return lp_fail(LP_ERR_INVALID, "lp_kernel_spectrum: PSF sides must be odd and >= 1 (got %d x %d)", hk, wk);
    if (prec != LP_PREC_FP32 && prec != LP_PREC_SPLIT_BF16)
        return lp_fail(LP_ERR_UNSUPPORTED, "lp_kernel_spectrum: precision %d is not built", (int)prec);
    const bool split = prec == LP_PREC_SPLIT_BF16;
    if (pad_ny < 0 || pad_nx < 0 || max_h < 0 || max_w < 0)
        return lp_fail(LP_ERR_INVALID, "lp_kernel_spectrum: negative size");
    int Ny = pad_ny, Nx = pad_nx;
    if (Ny == 0) {
        if (max_h < 1) return lp_fail(LP_ERR_INVALID, "lp_kernel_spectrum: need max_h or pad_ny");
        Ny = split ? tc_supported_size(max_h + hk - 1) : lp_supported_size(max_h + hk - 1);
        if (Ny < 0) return lp_fail(LP_ERR_UNSUPPORTED, "no supported FFT length >= %d", max_h + hk - 1);
    }
    if (Nx == 0) {
        if (max_w < 1) return lp_fail(LP_ERR_INVALID, "lp_kernel_spectrum: need max_w or pad_nx");
        Nx = lp_supported_size(max_w + wk - 1);
        if (Nx < 0) return lp_fail(LP_ERR_UNSUPPORTED, "no supported FFT length >= %d", max_w + wk - 1);
    }
    if (!find_size(Ny) || !find_size(Nx))
        return lp_fail(LP_ERR_UNSUPPORTED, "padded size %d x %d is not a supported FFT length", Ny, Nx);
    if (Ny < hk || Nx < wk)
        return lp_fail(LP_ERR_INVALID, "padded size %d x %d is smaller than the PSF %d x %d", Ny, Nx, hk, wk);
    if (split && find_size(Ny)->tc_smem == 0)
        return lp_fail(LP_ERR_UNSUPPORTED, "column length %d has no split-precision tensor-core pass", Ny);
    if (!fft64_supported(Ny) || !fft64_supported(Nx))
        return lp_fail(LP_ERR_UNSUPPORTED, "FP64 spectrum transform cannot factor %d x %d", Ny, Nx);

    DeviceGuard dg(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, K) != cudaSuccess || pa.type != cudaMemoryTypeDevice ||
        pa.device != ctx->device) {
        cudaGetLastError();
        return lp_fail(LP_ERR_INVALID, "lp_kernel_spectrum: K is not a device pointer of device %d", ctx->device);
    }
    // plans used later by lp_map (allocating here keeps lp_map allocation-free
    // once its workspace exists)
    const PlanRec* pr;
    lp_status s0 = lp_get_plan(ctx, Ny, &pr);
    if (s0 != LP_OK) return s0;
    s0 = lp_get_plan(ctx, Nx, &pr);
    if (s0 != LP_OK) return s0;

    // fingerprint + symmetry (one small device round trip); the third word
    // holds the flag of the value comparisons below
    unsigned long long* d_fp = nullptr;
    CUDA_TRY(cudaMallocAsync((void**)&d_fp, 24, st));
    CUDA_TRY(cudaMemsetAsync(d_fp, 0, 24, st));
    CUDA_TRY(psf_fingerprint_launch(K, (long long)hk * wk, d_fp, st));
    CUDA_TRY(psf_symmetry_launch(K, hk, wk, reinterpret_cast<int*>(d_fp + 1), st));
    unsigned long long host_fp[2] = {0, 0};
    CUDA_TRY(cudaMemcpyAsync(host_fp, d_fp, 16, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    const int is_real = (int)(host_fp[1] & 0xffffffffull) == 0;
    if (ctx->test_hook & LP_TEST_FP_COLLIDE) host_fp[0] = 0;
    const SpecKey key0{host_fp[0], hk, wk, Ny, Nx, (int)prec, 0};
    int* d_diff = reinterpret_cast<int*>(d_fp + 2);

    // Cached spectra of the same fingerprint and sizes, confirmed by comparing
    // K with each one's stored copy value by value (a fingerprint collision
    // never returns another PSF's spectrum).  Called with spec_mu held.
    auto find_cached = [&](lp_spectrum** hit, int* next_salt) -> lp_status {
        *hit = nullptr;
        *next_salt = 0;
        SpecKey lo = key0;
        lo.salt = -1;
        for (auto it = ctx->spectra.upper_bound(lo); it != ctx->spectra.end() && it->first.same_request(key0); ++it) {
            if (it->first.salt + 1 > *next_salt) *next_salt = it->first.salt + 1;
            int diff = 1;
            CUDA_TRY(cudaStreamWaitEvent(st, it->second->ready, 0));  // its copy of K is in place
            CUDA_TRY(cudaMemsetAsync(d_diff, 0, sizeof(int), st));
            CUDA_TRY(psf_compare_launch(K, it->second->kcopy, (long long)hk * wk, d_diff, st));
            CUDA_TRY(cudaMemcpyAsync(&diff, d_diff, sizeof(int), cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            if (diff == 0) {
                *hit = it->second;
                return LP_OK;
            }
        }
        return LP_OK;
    };
    lp_reap_released(ctx, false);
    int salt = 0;
    {
        std::lock_guard<std::mutex> g(ctx->spec_mu);
        lp_spectrum* hit = nullptr;
        const lp_status fs = find_cached(&hit, &salt);
        if (fs != LP_OK) {
            cudaFreeAsync(d_fp, st);
            return fs;
        }
        if (hit) {
            hit->refcount++;
            *out = hit;
            CUDA_TRY(cudaFreeAsync(d_fp, st));
            return LP_OK;
        }
    }
    const int ncols = Nx / 2 + 1;
    const long long ldK = ((long long)Ny + 31) / 32 * 32;
    const size_t bytes = (size_t)ncols * ldK * (is_real ? 4 : 8);
    auto spec = new (std::nothrow) lp_spectrum();
    if (!spec) {
        cudaFreeAsync(d_fp, st);
        return lp_fail(LP_ERR_OOM, "host allocation failed");
    }
    spec->ctx = ctx;
    spec->key = key0;
    spec->ny = Ny;
    spec->nx = Nx;
    spec->hk = hk;
    spec->wk = wk;
    spec->is_real = is_real;
    spec->prec = prec;
    spec->ldK = ldK;
    spec->bytes = bytes;
    spec->kbytes = sizeof(double) * (size_t)hk * wk;
    spec->refcount = 1;
    auto discard = [&](lp_spectrum* sp) {
        cudaStreamSynchronize(st);
        free_spectrum(ctx, sp);
    };
    void* dptr = nullptr;
    lp_status sa = lp_ctx_alloc(ctx, bytes, &dptr);
    if (sa == LP_OK) {
        spec->data = dptr;
        void* kc = nullptr;
        sa = lp_ctx_alloc(ctx, spec->kbytes, &kc);
        spec->kcopy = static_cast<double*>(kc);
    }
    if (sa != LP_OK) {
        const std::string msg = lp_last_error();
        cudaFreeAsync(d_fp, st);
        discard(spec);
        return lp_fail(sa, "%s", msg.c_str());
    }
    // FP64 scratch, stream-ordered, released right after the build
    const size_t w1 = sizeof(double2) * (size_t)hk * Nx;
    const size_t w2 = sizeof(double2) * (size_t)Ny * ncols;
    char* scratch = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&scratch, 2 * w1 + 2 * w2, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(d_fp, st);
        discard(spec);
        return lp_fail(LP_ERR_OOM, "spectrum scratch (%zu bytes): %s", 2 * w1 + 2 * w2, cudaGetErrorString(e));
    }
    e = cudaMemcpyAsync(spec->kcopy, K, spec->kbytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(dptr, 0, bytes, st);
    if (e == cudaSuccess)
        e = psf_spectrum_build(K, hk, wk, Ny, Nx, is_real, dptr, ldK, (double2*)scratch,
                               (double2*)(scratch + w1), (double2*)(scratch + 2 * w1),
                               (double2*)(scratch + 2 * w1 + w2), st);
    cudaFreeAsync(scratch, st);
    for (int i = 0; e == cudaSuccess && i < lp_spectrum::kUseSlots; ++i)
        e = cudaEventCreateWithFlags(&spec->use_event[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&spec->ready, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(spec->ready, st);
    if (e != cudaSuccess) {
        cudaFreeAsync(d_fp, st);
        discard(spec);
        return lp_fail(LP_ERR_CUDA, "spectrum build: %s", cudaGetErrorString(e));
    }
    {
        std::lock_guard<std::mutex> g(ctx->spec_mu);
        // another thread may have built the same PSF meanwhile
        lp_spectrum* hit = nullptr;
        const lp_status fs = find_cached(&hit, &salt);
        if (fs != LP_OK || hit) {
            if (hit) {
                hit->refcount++;
                *out = hit;
            }
            cudaFreeAsync(d_fp, st);
            discard(spec);
            return fs;
        }
        spec->key.salt = salt;
        ctx->spectra.emplace(spec->key, spec);
    }
    CUDA_TRY(cudaFreeAsync(d_fp, st));
    *out = spec;
    return LP_OK;
}

extern "C" lp_status lp_spectrum_info(const lp_spectrum* s, int* ny, int* nx, int* hk, int* wk,
                                      int* is_real)
{
    if (!s) return lp_fail(LP_ERR_INVALID, "lp_spectrum_info: NULL spectrum");
    if (ny) *ny = s->ny;
    if (nx) *nx = s->nx;
    if (hk) *hk = s->hk;
    if (wk) *wk = s->wk;
    if (is_real) *is_real = s->is_real;
    return LP_OK;
}

extern "C" lp_status lp_spectrum_copy(const lp_spectrum* s, float* dst, size_t dst_floats, void* stream)
{
    if (!s || !dst) return lp_fail(LP_ERR_INVALID, "lp_spectrum_copy: NULL argument");
    const size_t per = s->is_real ? 1 : 2;
    const size_t ncols = (size_t)s->nx / 2 + 1;
    if (dst_floats < ncols * s->ny * per)
        return lp_fail(LP_ERR_INVALID, "lp_spectrum_copy: destination holds %zu floats, need %zu",
                       dst_floats, ncols * s->ny * per);
    DeviceGuard dg(s->ctx->device);
    CUDA_TRY(cudaMemcpy2DAsync(dst, (size_t)s->ny * per * 4, s->data, (size_t)s->ldK * per * 4,
                               (size_t)s->ny * per * 4, ncols, cudaMemcpyDeviceToDevice,
                               static_cast<cudaStream_t>(stream)));
    return LP_OK;
}

static void free_spectrum(lp_ctx* ctx, lp_spectrum* s)
{
    lp_ctx_free(ctx, s->data, s->bytes);
    lp_ctx_free(ctx, s->kcopy, s->kbytes);
    if (s->ready) cudaEventDestroy(s->ready);
    for (int i = 0; i < lp_spectrum::kUseSlots; ++i)
        if (s->use_event[i]) cudaEventDestroy(s->use_event[i]);
    delete s;
}

// true when the spectrum's build and every recorded use have completed
static bool spectrum_idle(lp_spectrum* s, bool wait)
{
    if (s->use_overflow) {
        // used on more streams than it tracks: only a device-wide wait is sure
        if (!wait) return false;
        cudaDeviceSynchronize();
        return true;
    }
    cudaEvent_t evs[1 + lp_spectrum::kUseSlots];
    int n = 0;
    evs[n++] = s->ready;
    for (int i = 0; i < s->nuse; ++i) evs[n++] = s->use_event[i];
    for (int i = 0; i < n; ++i) {
        if (!evs[i]) continue;
        const cudaError_t q = wait ? cudaEventSynchronize(evs[i]) : cudaEventQuery(evs[i]);
        if (q == cudaErrorNotReady) return false;
        if (q != cudaSuccess) cudaGetLastError();  // a failed context: nothing is running any more
    }
    return true;
}

void lp_reap_released(lp_ctx* ctx, bool wait)
{
    std::lock_guard<std::mutex> g(ctx->spec_mu);
    if (ctx->released.empty()) return;
    DeviceGuard dg(ctx->device);
    std::vector<lp_spectrum*> keep;
    for (lp_spectrum* s : ctx->released) {
        if (spectrum_idle(s, wait)) free_spectrum(ctx, s);
        else keep.push_back(s);
    }
    ctx->released.swap(keep);
}

void lp_spectrum_ref(lp_ctx* ctx, const lp_spectrum* s)
{
    std::lock_guard<std::mutex> g(ctx->spec_mu);
    const_cast<lp_spectrum*>(s)->refcount++;
}

lp_status lp_spectrum_unref(lp_ctx* ctx, const lp_spectrum* cs)
{
    lp_spectrum* s = const_cast<lp_spectrum*>(cs);
    {
        std::lock_guard<std::mutex> g(ctx->spec_mu);
        auto it = ctx->spectra.find(s->key);
        if (it == ctx->spectra.end() || it->second != s)
            return lp_fail(LP_ERR_INVALID, "lp_spectrum_release: unknown spectrum");
        if (--s->refcount > 0) return LP_OK;
        // no new map can name it any more; maps already enqueued may still
        // read it, so it is freed only once their use events have completed
        ctx->spectra.erase(it);
        ctx->released.push_back(s);
    }
    lp_reap_released(ctx, false);
    return LP_OK;
}

extern "C" lp_status lp_spectrum_release(lp_ctx* ctx, lp_spectrum* s)
{
    if (!ctx || !s) return lp_fail(LP_ERR_INVALID, "lp_spectrum_release: NULL argument");
    if (s->ctx != ctx) return lp_fail(LP_ERR_INVALID, "lp_spectrum_release: spectrum belongs to another context");
    return lp_spectrum_unref(ctx, s);
}

lp_status lp_wait_spectra_built(const lp_spectrum* const* spectra, int n, cudaStream_t st)
{
    for (int k = 0; k < n; ++k) {
        lp_spectrum* s = const_cast<lp_spectrum*>(spectra[k]);
        if (s->built.load(std::memory_order_acquire)) continue;
        const cudaError_t q = cudaEventQuery(s->ready);
        if (q == cudaSuccess) {
            s->built.store(true, std::memory_order_release);
        } else if (q == cudaErrorNotReady) {
            CUDA_TRY(cudaStreamWaitEvent(st, s->ready, 0));
        } else {
            return lp_fail(LP_ERR_CUDA, "spectrum build: %s", cudaGetErrorString(q));
        }
    }
    return LP_OK;
}

void lp_note_spectra_used(lp_ctx* ctx, const lp_spectrum* const* spectra, int n, cudaStream_t st)
{
    std::lock_guard<std::mutex> g(ctx->spec_mu);
    for (int k = 0; k < n; ++k) {
        lp_spectrum* s = const_cast<lp_spectrum*>(spectra[k]);
        int slot = -1;
        for (int i = 0; i < s->nuse; ++i)
            if (s->use_stream[i] == st) slot = i;
        if (slot < 0) {
            if (s->nuse == lp_spectrum::kUseSlots) {
                s->use_overflow = true;
                continue;
            }
            slot = s->nuse++;
            s->use_stream[slot] = st;
        }
        if (cudaEventRecord(s->use_event[slot], st) != cudaSuccess) {
            cudaGetLastError();
            s->use_overflow = true;
        }
    }
}

// ---------------------------------------------------------------------------
// map
// ---------------------------------------------------------------------------
static inline long long even_up(long long x) { return (x + 1) / 2 * 2; }

// workspace layout: T (ncolsT x ldT) then U (n x ncolsU x ldU), complex64,
// both column-blocked
static void map_dims(int h, int w, int ny, int nx, int hk, int wk, lp_outmode mode, MapDims* d)
{
    d->ncols = nx / 2 + 1;
    d->ncolsT = t_cols_alloc(d->ncols);
    d->ncolsU = u_cols_alloc(d->ncols);
    d->ldT = even_up(h);
    if (mode == LP_OUT_FULL) {
        d->Hout = h + hk - 1;
        d->Wout = w + wk - 1;
        d->r0 = ny - (hk - 1) / 2;
        d->c0 = nx - (wk - 1) / 2;
        if (d->r0 == ny) d->r0 = 0;
        if (d->c0 == nx) d->c0 = 0;
    } else {
        d->Hout = h;
        d->Wout = w;
        d->r0 = 0;
        d->c0 = 0;
    }
    d->ldU = even_up(d->Hout);
    d->prec = (int)LP_PREC_FP32;
    d->ny = ny;
    const SizeKernels* k = find_size(ny);
    d->batch = (k && k->batch) ? 1 : 0;
}

size_t lp_park_bytes(const MapDims& d) { return 8ull * (size_t)d.ncols * (size_t)d.ny; }

// the batched column pass parks its forward column spectra in the workspace
// where they do not fit shared memory next to the exchange buffer
static inline bool uses_park(const MapDims& d, int nchunk)
{
    const SizeKernels* k = find_size(d.ny);
    const bool global_park = k && (long long)k->smem_bytes + 8ll * d.ny > 227ll * 1024;
    return nchunk > 1 && d.batch && global_park && d.prec == (int)LP_PREC_FP32;
}

size_t lp_workspace_bytes(const MapDims& d, int n)
{
    const int nchunk = n < kMaxSpectraPerLaunch ? n : kMaxSpectraPerLaunch;
    return 8ull * ((size_t)d.ncolsT * (size_t)d.ldT + (size_t)d.ncolsU * (size_t)nchunk * (size_t)d.ldU) +
           (uses_park(d, nchunk) ? lp_park_bytes(d) + 256 : 0) + 256;
}

extern "C" size_t lp_map_workspace_bytes(int h, int w, int ny, int nx, int hk, int wk, int n,
                                         lp_outmode mode)
{
    if (h < 1 || w < 1 || ny < 1 || nx < 1 || n < 1 || hk < 1 || wk < 1) return 0;
    MapDims d;
    map_dims(h, w, ny, nx, hk, wk, mode, &d);
    return lp_workspace_bytes(d, n);
}

// Checks shared by every map entry point.  need_pad: the spectra's padded
// size must hold the whole linear convolution of the map (Sec. 2.5); the
// tiled map instead needs spectra of one PSF size (its tile geometry).
static lp_status validate_map_args(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                                   const lp_spectrum* const* spectra, int n, const void* out, lp_outmode mode,
                                   lp_precision prec, bool need_pad)
{
    if (!ctx || !L || !spectra || !out) return lp_fail(LP_ERR_INVALID, "lp_map: NULL argument");
    if (h < 1 || w < 1) return lp_fail(LP_ERR_INVALID, "lp_map: empty map %d x %d", h, w);
    if (ldl < w) return lp_fail(LP_ERR_INVALID, "lp_map: ldl %d < w %d", ldl, w);
    if (n < 1) return lp_fail(LP_ERR_INVALID, "lp_map: need at least one spectrum");
    if (mode != LP_OUT_SAME && mode != LP_OUT_FULL) return lp_fail(LP_ERR_INVALID, "lp_map: bad output mode");
    if (prec != LP_PREC_FP32 && prec != LP_PREC_SPLIT_BF16)
        return lp_fail(LP_ERR_UNSUPPORTED, "lp_map: precision %d is not built", (int)prec);
    const lp_spectrum* s0 = spectra[0];
    if (!s0) return lp_fail(LP_ERR_INVALID, "lp_map: spectrum 0 is NULL");
    for (int k = 0; k < n; ++k) {
        const lp_spectrum* s = spectra[k];
        if (!s) return lp_fail(LP_ERR_INVALID, "lp_map: spectrum %d is NULL", k);
        if (s->ctx != ctx) return lp_fail(LP_ERR_INVALID, "lp_map: spectrum %d belongs to another context", k);
        if (s->ny != s0->ny || s->nx != s0->nx)
            return lp_fail(LP_ERR_INVALID, "lp_map: spectra differ in padded size (%dx%d vs %dx%d)", s->ny,
                           s->nx, s0->ny, s0->nx);
        if (!need_pad && (s->hk != s0->hk || s->wk != s0->wk))
            return lp_fail(LP_ERR_INVALID, "lp_map_tiled: spectra of different PSF sizes");
        if (need_pad && (s->ny < h + s->hk - 1 || s->nx < w + s->wk - 1))
            return lp_fail(LP_ERR_INVALID,
                           "lp_map: spectrum %d padded to %d x %d, the map %d x %d with a %d x %d PSF "
                           "needs >= %d x %d",
                           k, s->ny, s->nx, h, w, s->hk, s->wk, h + s->hk - 1, w + s->wk - 1);
        if (mode == LP_OUT_FULL && (s->hk != s0->hk || s->wk != s0->wk))
            return lp_fail(LP_ERR_INVALID, "lp_map: FULL output needs spectra of equal PSF size");
        if (s->prec != prec) return lp_fail(LP_ERR_INVALID, "lp_map: spectrum %d has another precision", k);
    }
    if (prec == LP_PREC_SPLIT_BF16 && find_size(s0->ny)->tc_smem == 0)
        return lp_fail(LP_ERR_UNSUPPORTED, "lp_map: column length %d has no split-precision pass", s0->ny);
    return LP_OK;
}

lp_status lp_validate_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                          const lp_spectrum* const* spectra, int n, const void* out, int ldo,
                          lp_outmode mode, lp_precision prec, MapDims* d)
{
    const lp_status st = validate_map_args(ctx, L, h, w, ldl, spectra, n, out, mode, prec, true);
    if (st != LP_OK) return st;
    const lp_spectrum* s0 = spectra[0];
    map_dims(h, w, s0->ny, s0->nx, s0->hk, s0->wk, mode, d);
    d->prec = (int)prec;
    if (ldo < d->Wout) return lp_fail(LP_ERR_INVALID, "lp_map: ldo %d < output width %d", ldo, d->Wout);
    return LP_OK;
}

// Declared extents for the debug builds' bounds checks: T holds ncolsT x ldT
// complex elements; LP_TEST_BOUNDS declares it one column block short, so
// that the checks of the units touching the last columns fire (the
// accesses stay inside the real buffer: nothing out of bounds happens).
static long long t_extent(const lp_ctx* ctx, const MapDims& d)
{
    const long long cols = (ctx->test_hook.load() & LP_TEST_BOUNDS) ? d.ncolsT - 2 : d.ncolsT;
    return cols * d.ldT;
}

static long long k_extent(const lp_spectrum* s) { return (long long)(s->bytes / (s->is_real ? 4 : 8)); }

// The three passes as separate launches (row pairs [pair0, pair1) for the
// row passes), composed by lp_launch_map and by the banded host-buffer map.
static lp_status launch_rows_forward(lp_ctx* ctx, const PlanRec* px, const float* L, int h, int w, int ldl,
                                     const MapDims& d, float2* T, int pair0, int pair1, cudaStream_t st)
{
    P1Args a1;
    a1.L = L;
    a1.ldl = ldl;
    a1.H = h;
    a1.W = w;
    a1.Wst = (w + 3) / 4 * 4;
    a1.vec16 = ((reinterpret_cast<uintptr_t>(L) & 15) == 0 && ldl % 4 == 0 && w % 4 == 0) ? 1 : 0;
    a1.T = T;
    a1.ldT = d.ldT;
    a1.pair0 = pair0;
    a1.npairs = pair1;
    a1.ncols = d.ncols;
    a1.tw = px->fwd;
    a1.err = ctx->d_err;
    a1.t_elems = t_extent(ctx, d);
    const int tok = lp_pass_begin(ctx, 0, st);
    CUDA_TRY(px->k->p1(a1, st));
    lp_pass_end(ctx, tok, st);
    return LP_OK;
}

// Column distance of the column pass's T prefetch: about one wave of
// resident blocks (three per SM), computed once per context.
static int prefetch_ahead(lp_ctx* ctx)
{
    if (ctx->sms == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess) sms = 0;
        ctx->sms = sms > 0 ? sms : -1;
    }
    return ctx->sms > 0 ? 3 * ctx->sms : 0;
}

// column pass for spectra [base, base+cnt) into U (cnt blocks of ncols x ldU)
static lp_status launch_columns(lp_ctx* ctx, const PlanRec* py, const lp_spectrum* const* spectra, int base,
                                int cnt, int h, const MapDims& d, const float2* T, float2* U, float2* park,
                                cudaStream_t st)
{
    const lp_spectrum* s0 = spectra[0];
    if (d.prec == (int)LP_PREC_SPLIT_BF16) {
        // tensor-core column pass: one launch per spectrum
        for (int i = 0; i < cnt; ++i) {
            P2TcArgs a2;
            P2Args& b = a2.a;
            b.T = T;
            b.ldT = d.ldT;
            b.H = h;
            for (int q = 0; q < kMaxSpectraPerLaunch; ++q) b.K[q] = nullptr;
            b.K[0] = spectra[base + i]->data;
            b.ldK = s0->ldK;
            b.nspec = 1;
            b.U = U + (size_t)i * d.ncolsU * d.ldU;
            b.ldU = d.ldU;
            b.specU = (long long)d.ncolsU * d.ldU;
            b.r0 = d.r0;
            b.Hout = d.Hout;
            b.HoutPad = (int)d.ldU;
            b.ncols = d.ncols;
            b.twf = py->fwd;
            b.twi = py->rev;
            b.park = nullptr;
            b.ahead = 0;
            b.err = ctx->d_err;
            b.t_elems = t_extent(ctx, d);
            b.u_elems = (long long)d.ncolsU * d.ldU;
            b.k_elems = k_extent(spectra[base + i]);
            b.park_elems = 0;
            a2.tables = static_cast<const uint4*>(py->tc_tables);
            a2.err = ctx->d_err;
            a2.no_mma = (ctx->test_hook & LP_TEST_TC_NO_MMA) ? 1 : 0;
            const int tok = lp_pass_begin(ctx, 1, st);
            CUDA_TRY(py->k->p2tc(a2, spectra[base + i]->is_real != 0, st));
            lp_pass_end(ctx, tok, st);
        }
        return LP_OK;
    }
    // the real-spectrum kernel needs every spectrum of the launch real:
    // split the chunk by kind
    int k0 = 0;
    while (k0 < cnt) {
        const int kind = spectra[base + k0]->is_real;
        int k1 = k0;
        while (k1 < cnt && spectra[base + k1]->is_real == kind) ++k1;
        P2Args a2;
        a2.T = T;
        a2.ldT = d.ldT;
        a2.H = h;
        for (int i = 0; i < kMaxSpectraPerLaunch; ++i)
            a2.K[i] = (i < k1 - k0) ? spectra[base + k0 + i]->data : nullptr;
        a2.ldK = s0->ldK;
        a2.nspec = k1 - k0;
        a2.U = U + (size_t)k0 * d.ncolsU * d.ldU;
        a2.ldU = d.ldU;
        a2.specU = (long long)d.ncolsU * d.ldU;
        a2.r0 = d.r0;
        a2.Hout = d.Hout;
        a2.HoutPad = (int)d.ldU;
        a2.ncols = d.ncols;
        a2.twf = py->fwd;
        a2.twi = py->rev;
        a2.park = park;
        a2.ahead = prefetch_ahead(ctx);
        a2.err = ctx->d_err;
        a2.t_elems = t_extent(ctx, d);
        a2.u_elems = (long long)(cnt - k0) * d.ncolsU * d.ldU;
        a2.k_elems = k_extent(spectra[base + k0]);
        for (int i = k0 + 1; i < k1; ++i) a2.k_elems = std::min(a2.k_elems, k_extent(spectra[base + i]));
        a2.park_elems = park ? (long long)(lp_park_bytes(d) / 8) : 0;
        const int tok = lp_pass_begin(ctx, 1, st);
        CUDA_TRY(py->k->p2(a2, kind != 0, st));
        lp_pass_end(ctx, tok, st);
        k0 = k1;
    }
    return LP_OK;
}

static lp_status launch_rows_inverse(lp_ctx* ctx, const PlanRec* px, const MapDims& d, const float2* U, int cnt,
                                     float* const* out, int ldo, int pair0, int pair1, cudaStream_t st)
{
    P3Args a3;
    a3.U = U;
    a3.ldU = d.ldU;
    a3.specU = (long long)d.ncolsU * d.ldU;
    a3.Hout = d.Hout;
    a3.pair0 = pair0;
    a3.npairs = pair1;
    for (int i = 0; i < kMaxSpectraPerLaunch; ++i) a3.out[i] = i < cnt ? out[i] : nullptr;
    a3.ldo = ldo;
    a3.c0 = d.c0;
    a3.Wout = d.Wout;
    a3.ncols = d.ncols;
    a3.tw = px->rev;
    a3.err = ctx->d_err;
    a3.u_elems = (long long)cnt * d.ncolsU * d.ldU;
    const int tok = lp_pass_begin(ctx, 2, st);
    CUDA_TRY(px->k->p3(a3, cnt, st));
    lp_pass_end(ctx, tok, st);
    return LP_OK;
}

// park area after U in a workspace (256-byte aligned)
static inline float2* park_of(const MapDims& d, float2* U, int nchunk)
{
    const uintptr_t p = reinterpret_cast<uintptr_t>(U + (size_t)d.ncolsU * d.ldU * (size_t)nchunk);
    return reinterpret_cast<float2*>((p + 255) / 256 * 256);
}

// Launch P1, P2, P3 for n spectra (the validated sequence of lp_map).
lp_status lp_launch_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                        const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                        const MapDims& d, void* ws, cudaStream_t st)
{
    const lp_spectrum* s0 = spectra[0];
    const PlanRec *py, *px;
    lp_status ps = lp_get_plan(ctx, s0->ny, &py);
    if (ps != LP_OK) return ps;
    ps = lp_get_plan(ctx, s0->nx, &px);
    if (ps != LP_OK) return ps;
    float2* T = static_cast<float2*>(ws);
    float2* U = T + (size_t)d.ncolsT * d.ldT;
    const int nchunk = n < kMaxSpectraPerLaunch ? n : kMaxSpectraPerLaunch;
    float2* park = uses_park(d, nchunk) ? park_of(d, U, nchunk) : nullptr;
    // Inside a stream capture (a CUDA graph) the map may only launch
    // kernels: no spectrum build may still be pending (a wait on it would tie
    // the graph to that one build), no pass events, and no use events (the
    // library does not see the graph's replays; the caller keeps the spectra
    // alive while the graph may run).
    const bool capturing = lp_stream_capturing(st);
    if (capturing) {
        for (int k = 0; k < n; ++k)
            if (!spectra[k]->built.load(std::memory_order_acquire) && cudaEventQuery(spectra[k]->ready) != cudaSuccess)
                return lp_fail(LP_ERR_INVALID, "spectrum %d is still being built: synchronise before capturing", k);
        std::lock_guard<std::mutex> g(ctx->tim_mu);
        if (ctx->timing) return lp_fail(LP_ERR_INVALID, "pass timing is on: switch it off before capturing");
    } else if ((ps = lp_wait_spectra_built(spectra, n, st)) != LP_OK) {
        return ps;
    }
    if ((ps = launch_rows_forward(ctx, px, L, h, w, ldl, d, T, 0, (int)(d.ldT / 2), st)) != LP_OK) return ps;
    for (int base = 0; base < n; base += kMaxSpectraPerLaunch) {
        const int cnt = (n - base) < kMaxSpectraPerLaunch ? (n - base) : kMaxSpectraPerLaunch;
        if ((ps = launch_columns(ctx, py, spectra, base, cnt, h, d, T, U, park, st)) != LP_OK) return ps;
        if ((ps = launch_rows_inverse(ctx, px, d, U, cnt, out + base, ldo, 0, (int)(d.ldU / 2), st)) != LP_OK)
            return ps;
    }
    // recorded after the last pass (an event between the passes would stop
    // the next pass's launch from overlapping the previous one's tail)
    if (!capturing) lp_note_spectra_used(ctx, spectra, n, st);
    return LP_OK;
}

extern "C" lp_status lp_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                            const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                            lp_outmode mode, lp_precision prec, void* stream)
{
    MapDims d;
    lp_status st = lp_validate_map(ctx, L, h, w, ldl, spectra, n, out, ldo, mode, prec, &d);
    if (st != LP_OK) return st;
    for (int k = 0; k < n; ++k) {
        if (!out[k]) return lp_fail(LP_ERR_INVALID, "lp_map: out[%d] is NULL", k);
        const char* o0 = reinterpret_cast<const char*>(out[k]);
        const char* o1 = o0 + 4ull * ((size_t)(d.Hout - 1) * ldo + d.Wout);
        const char* l0 = reinterpret_cast<const char*>(L);
        const char* l1 = l0 + 4ull * ((size_t)(h - 1) * ldl + w);
        if (o0 < l1 && l0 < o1) return lp_fail(LP_ERR_INVALID, "lp_map: out[%d] overlaps L", k);
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!lp_stream_capturing(s)) lp_reap_released(ctx, false);  // frees memory: not inside a capture
    const lp_spectrum* s0 = spectra[0];
    void* ws = nullptr;
    st = lp_get_workspace(ctx, s, lp_map_workspace_bytes(h, w, s0->ny, s0->nx, s0->hk, s0->wk, n, mode), &ws);
    if (st != LP_OK) return st;
    return lp_launch_map(ctx, L, h, w, ldl, spectra, n, out, ldo, d, ws, s);
}

// Maps larger than the spectra's padded size: overlap-save tiles.  Sec. 4
// computes extended regions band by band; here the pieces share one grid,
// and each carries the PSF's reach around it as margin so that its pixels
// see every source within the PSF.  Output tile rows [a, a + th) of the SAME
// result need the input rows [a - cy, a + th + cy) (cy = (hk - 1) / 2),
// clipped to the map (rows outside it are zero).  In the Ny-point circular
// convolution of that window the tile's rows receive no wrapped-around term
// when Ny >= th + 2 cy: the tile starts r0 <= cy rows into the window and
// the window ends at most th + cy rows after the tile's start, so a kept
// output row o and an input row i of the window satisfy |o - i| <= th + cy
// - 1, and o - i +- Ny never falls within the PSF's support [-cy, cy].
// Hence th = Ny - (hk - 1) (hk = 2 cy + 1), and tw = Nx - (wk - 1) alike.
// A dimension the map covers in one tile has no margin beyond the map:
// there |o - i| <= h - 1, so h <= Ny - cy suffices (the SAME crop's own
// padding rule, tighter than h + hk - 1).  Each tile is one P1 / P2 / P3 sequence on the
// window (row and column offsets of the crop r0 = a - window start,
// c0 alike), writing its tile of out[] in place; tiles run in stream order
// and share one workspace.
extern "C" lp_status lp_map_tiled(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                                  const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                                  lp_precision prec, void* stream)
{
    lp_status st = validate_map_args(ctx, L, h, w, ldl, spectra, n, out, LP_OUT_SAME, prec, false);
    if (st != LP_OK) return st;
    if (ldo < w) return lp_fail(LP_ERR_INVALID, "lp_map_tiled: ldo %d < output width %d", ldo, w);
    const lp_spectrum* s0 = spectra[0];
    const int ny = s0->ny, nx = s0->nx, hk = s0->hk, wk = s0->wk;
    const int cy = (hk - 1) / 2, cx = (wk - 1) / 2;
    // one tile where the whole dimension fits (h <= Ny - cy), else tiles of
    // Ny - (hk - 1)
    const int th = h <= ny - cy ? h : ny - (hk - 1), tw = w <= nx - cx ? w : nx - (wk - 1);
    if (th < 1 || tw < 1)
        return lp_fail(LP_ERR_INVALID, "lp_map_tiled: padded size %d x %d leaves no tile for a %d x %d PSF", ny, nx,
                       hk, wk);
    for (int k = 0; k < n; ++k) {
        if (!out[k]) return lp_fail(LP_ERR_INVALID, "lp_map_tiled: out[%d] is NULL", k);
        const char* o0 = reinterpret_cast<const char*>(out[k]);
        const char* o1 = o0 + 4ull * ((size_t)(h - 1) * ldo + w);
        const char* l0 = reinterpret_cast<const char*>(L);
        const char* l1 = l0 + 4ull * ((size_t)(h - 1) * ldl + w);
        if (o0 < l1 && l0 < o1) return lp_fail(LP_ERR_INVALID, "lp_map_tiled: out[%d] overlaps L", k);
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (!lp_stream_capturing(s)) lp_reap_released(ctx, false);  // frees memory: not inside a capture
    // one workspace for the largest tile: window min(h, th + 2 cy) x
    // min(w, tw + 2 cx), min(h, th) kept rows
    MapDims dmax;
    map_dims(std::min(h, th + 2 * cy), std::min(w, tw + 2 * cx), ny, nx, hk, wk, LP_OUT_SAME, &dmax);
    dmax.Hout = std::min(h, th);
    dmax.ldU = even_up(dmax.Hout);
    dmax.prec = (int)prec;
    void* ws = nullptr;
    if ((st = lp_get_workspace(ctx, s, lp_workspace_bytes(dmax, n), &ws)) != LP_OK) return st;
    std::vector<float*> o(n);
    for (int a = 0; a < h; a += th) {
        const int ra = std::max(0, a - cy), rb = std::min(h, a + th + cy);
        for (int b = 0; b < w; b += tw) {
            const int ca = std::max(0, b - cx), cb = std::min(w, b + tw + cx);
            MapDims d;
            map_dims(rb - ra, cb - ca, ny, nx, hk, wk, LP_OUT_SAME, &d);
            d.Hout = std::min(th, h - a);
            d.Wout = std::min(tw, w - b);
            d.r0 = a - ra;
            d.c0 = b - ca;
            d.ldU = even_up(d.Hout);
            d.prec = (int)prec;
            for (int k = 0; k < n; ++k) o[k] = out[k] + (size_t)a * ldo + b;
            st = lp_launch_map(ctx, L + (size_t)ra * ldl + ca, rb - ra, cb - ca, ldl, spectra, n, o.data(), ldo, d,
                               ws, s);
            if (st != LP_OK) return st;
        }
    }
    return LP_OK;
}

// Host-buffer map, pipelined in row bands: the map is copied up band by band
// on an internal stream while the row pass transforms the bands already on
// the device, and the output is copied down band by band while the inverse
// row pass produces the next bands.  The column pass needs every row, so it
// runs between the two.  Everything is ordered after the caller's stream at
// entry, and the caller's stream waits for the last copy at exit.
static constexpr int kHostBands = 8;

// Bands of a host map's upload or download: each copy costs a fixed
// overhead, so bands are at least ~32 MB (2 to kHostBands of them).
// Measured end to end on the 4096^2 map (67 MB each way): 8 bands 34.7K,
// 4 bands 37.5K, 2 bands 37.9K Mpix/s.
static int host_bands(size_t bytes, int npairs)
{
    long long nb = (long long)(bytes / (32ull << 20));
    if (nb < 2) nb = 2;
    if (nb > kHostBands) nb = kHostBands;
    return npairs < nb ? npairs : (int)nb;
}

static lp_status host_streams(lp_ctx* ctx)
{
    if (ctx->hs_in) return LP_OK;
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->hs_in, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->hs_out, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamCreateWithFlags(&ctx->hs_comp, cudaStreamNonBlocking));
    for (auto& ev : ctx->hs_ofree) CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    for (int i = 0; i < 2 * kHostBands + 2; ++i) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->hs_events.push_back(e);
    }
    for (auto& ev : ctx->hs_lfree) CUDA_TRY(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    return LP_OK;
}

extern "C" lp_status lp_map_host(lp_ctx* ctx, const float* L_host, int h, int w, int ldl,
                                 const lp_spectrum* const* spectra, int n, float* const* out_host,
                                 int ldo, lp_outmode mode, lp_precision prec, void* stream)
{
    MapDims d;
    lp_status st = lp_validate_map(ctx, L_host, h, w, ldl, spectra, n, out_host, ldo, mode, prec, &d);
    if (st != LP_OK) return st;
    for (int k = 0; k < n; ++k)
        if (!out_host[k]) return lp_fail(LP_ERR_INVALID, "lp_map_host: out[%d] is NULL", k);
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (lp_stream_capturing(s))
        return lp_fail(LP_ERR_INVALID, "lp_map_host: host copies on internal streams cannot be captured");
    const lp_spectrum* s0 = spectra[0];
    const PlanRec *py, *px;
    if ((st = lp_get_plan(ctx, s0->ny, &py)) != LP_OK) return st;
    if ((st = lp_get_plan(ctx, s0->nx, &px)) != LP_OK) return st;
    // staging: two maps L (h x w, packed), then two sets of n outputs
    // (Hout x Wout, packed); both alternate between calls, so that a map's
    // upload need not wait for the previous map's row pass
    const size_t lbytes = 4ull * (size_t)h * w;
    const size_t obytes = 4ull * (size_t)d.Hout * d.Wout;
    const size_t lb = (lbytes + 255) / 256 * 256, ob = (obytes + 255) / 256 * 256;
    const size_t need = 2ull * lb + 2ull * (size_t)n * ob;
    std::lock_guard<std::mutex> host_lock(ctx->host_mu);  // one host map enqueued at a time per context
    {
        std::lock_guard<std::mutex> g(ctx->ws_mu);
        if (ctx->staging_bytes < need) {
            if (ctx->staging) {
                // only the context's host-map streams touch the staging buffers
                for (cudaStream_t hs : {ctx->hs_in, ctx->hs_comp, ctx->hs_out})
                    if (hs) cudaStreamSynchronize(hs);
                lp_ctx_free(ctx, ctx->staging, ctx->staging_bytes);
                ctx->staging = nullptr;
                ctx->staging_bytes = 0;
            }
            void* p = nullptr;
            st = lp_ctx_alloc(ctx, need, &p);
            if (st != LP_OK) return st;
            ctx->staging = p;
            ctx->staging_bytes = need;
            ctx->hs_lfree_valid[0] = ctx->hs_lfree_valid[1] = false;
            ctx->hs_ofree_valid[0] = ctx->hs_ofree_valid[1] = false;
        }
    }
    if ((st = host_streams(ctx)) != LP_OK) return st;
    cudaStream_t c = ctx->hs_comp;  // the passes of host maps run here, with their own workspace
    const int obuf = ctx->hs_obuf, lbuf = ctx->hs_lbuf;
    char* base = static_cast<char*>(ctx->staging);
    float* dL = reinterpret_cast<float*>(base + (size_t)lbuf * lb);
    std::vector<float*> dout(n);
    for (int k = 0; k < n; ++k) dout[k] = reinterpret_cast<float*>(base + 2 * lb + ((size_t)obuf * n + k) * ob);
    void* ws = nullptr;
    st = lp_get_workspace(ctx, c, lp_map_workspace_bytes(h, w, s0->ny, s0->nx, s0->hk, s0->wk, n, mode), &ws);
    if (st != LP_OK) return st;
    float2* T = static_cast<float2*>(ws);
    float2* U = T + (size_t)d.ncolsT * d.ldT;
    const int nchunk = n < kMaxSpectraPerLaunch ? n : kMaxSpectraPerLaunch;
    float2* park = uses_park(d, nchunk) ? park_of(d, U, nchunk) : nullptr;
    cudaEvent_t* ev = ctx->hs_events.data();
    cudaEvent_t ev_start = ev[0], ev_end = ev[1];
    cudaEvent_t* ev_in = ev + 2;                 // kHostBands
    cudaEvent_t* ev_out = ev + 2 + kHostBands;   // kHostBands
    cudaEvent_t ev_lfree = ctx->hs_lfree[lbuf];

    // Ordering.  The upload waits until the row pass of the host map two back
    // (the last one that used this input staging buffer) has read it (the
    // first time: for the caller's earlier work on the stream).  The passes wait only for their input bands, the spectra's
    // builds, and -- before writing output staging buffer b -- the download
    // of the call two back that used b; so a map's passes overlap the
    // previous map's download.  The download waits for the caller's earlier
    // work on the stream (it writes caller memory), and the caller's stream
    // waits for the download, so the stream reaches the end of this call only
    // with every output in host memory.
    CUDA_TRY(cudaEventRecord(ev_start, s));
    if (ctx->hs_lfree_valid[lbuf]) CUDA_TRY(cudaStreamWaitEvent(ctx->hs_in, ev_lfree, 0));
    else CUDA_TRY(cudaStreamWaitEvent(ctx->hs_in, ev_start, 0));
    CUDA_TRY(cudaStreamWaitEvent(ctx->hs_out, ev_start, 0));
    for (int k = 0; k < n; ++k) CUDA_TRY(cudaStreamWaitEvent(c, spectra[k]->ready, 0));

    const int npairs = (int)(d.ldT / 2);
    const int nb_in = host_bands(lbytes, npairs);
    for (int b = 0; b < nb_in; ++b) {
        const int q0 = (int)((long long)npairs * b / nb_in), q1 = (int)((long long)npairs * (b + 1) / nb_in);
        const int r0 = 2 * q0, r1 = (2 * q1 < h) ? 2 * q1 : h;
        if (r1 > r0)
            CUDA_TRY(cudaMemcpy2DAsync(dL + (size_t)r0 * w, 4ull * w, L_host + (size_t)r0 * ldl, 4ull * ldl,
                                       4ull * w, r1 - r0, cudaMemcpyHostToDevice, ctx->hs_in));
        CUDA_TRY(cudaEventRecord(ev_in[b], ctx->hs_in));
        CUDA_TRY(cudaStreamWaitEvent(c, ev_in[b], 0));
        if ((st = launch_rows_forward(ctx, px, dL, h, w, w, d, T, q0, q1, c)) != LP_OK) return st;
    }
    CUDA_TRY(cudaEventRecord(ev_lfree, c));  // this input staging map may be overwritten after this
    ctx->hs_lfree_valid[lbuf] = true;
    ctx->hs_lbuf = lbuf ^ 1;
    const int opairs = (int)(d.ldU / 2);
    const int nb_out = host_bands(obytes * (size_t)n, opairs);
    for (int cb = 0; cb < n; cb += kMaxSpectraPerLaunch) {
        const int cnt = (n - cb) < kMaxSpectraPerLaunch ? (n - cb) : kMaxSpectraPerLaunch;
        if ((st = launch_columns(ctx, py, spectra, cb, cnt, h, d, T, U, park, c)) != LP_OK) return st;
        if (cb == 0 && ctx->hs_ofree_valid[obuf]) CUDA_TRY(cudaStreamWaitEvent(c, ctx->hs_ofree[obuf], 0));
        for (int b = 0; b < nb_out; ++b) {
            const int q0 = (int)((long long)opairs * b / nb_out), q1 = (int)((long long)opairs * (b + 1) / nb_out);
            if ((st = launch_rows_inverse(ctx, px, d, U, cnt, dout.data() + cb, d.Wout, q0, q1, c)) != LP_OK)
                return st;
            CUDA_TRY(cudaEventRecord(ev_out[b], c));
            CUDA_TRY(cudaStreamWaitEvent(ctx->hs_out, ev_out[b], 0));
            const int r0 = 2 * q0, r1 = (2 * q1 < d.Hout) ? 2 * q1 : d.Hout;
            if (r1 <= r0) continue;
            for (int k = cb; k < cb + cnt; ++k)
                CUDA_TRY(cudaMemcpy2DAsync(out_host[k] + (size_t)r0 * ldo, 4ull * ldo, dout[k] + (size_t)r0 * d.Wout,
                                           4ull * d.Wout, 4ull * d.Wout, r1 - r0, cudaMemcpyDeviceToHost,
                                           ctx->hs_out));
        }
    }
    lp_note_spectra_used(ctx, spectra, n, c);
    CUDA_TRY(cudaEventRecord(ctx->hs_ofree[obuf], ctx->hs_out));
    ctx->hs_ofree_valid[obuf] = true;
    ctx->hs_obuf = obuf ^ 1;
    CUDA_TRY(cudaEventRecord(ev_end, ctx->hs_out));
    CUDA_TRY(cudaStreamWaitEvent(s, ev_end, 0));
    return LP_OK;
}

extern "C" lp_status lp_set_test_hook(lp_ctx* ctx, int hook)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_set_test_hook: NULL context");
    if (hook & ~(LP_TEST_TC_NO_MMA | LP_TEST_FP_COLLIDE | LP_TEST_SERVE_FAIL | LP_TEST_BOUNDS))
        return lp_fail(LP_ERR_INVALID, "lp_set_test_hook: unknown hook 0x%x", hook);
    ctx->test_hook = hook;
    return LP_OK;
}

extern "C" lp_status lp_sync_status(lp_ctx* ctx, void* stream, int timeout_ms)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_sync_status: NULL context");
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t q = cudaStreamQuery(s);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady)
            return lp_fail(LP_ERR_CUDA, "lp_sync_status: %s", cudaGetErrorString(q));
        if (timeout_ms >= 0) {
            const auto el = std::chrono::duration_cast<std::chrono::milliseconds>(
                std::chrono::steady_clock::now() - t0).count();
            if (el >= timeout_ms) return lp_fail(LP_ERR_TIMEOUT, "lp_sync_status: stream busy after %d ms", timeout_ms);
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    lp_reap_released(ctx, false);
    int herr = 0;
    CUDA_TRY(cudaMemcpy(&herr, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != 0) {
        CUDA_TRY(cudaMemset(ctx->d_err, 0, sizeof(int)));
        return lp_fail(LP_ERR_DEVICE, "lp_sync_status: device status word 0x%x", herr);
    }
    return LP_OK;
}

// ---------------------------------------------------------------------------
// Eq. (4): several source classes
// ---------------------------------------------------------------------------
extern "C" lp_status lp_map_multiclass(lp_ctx* ctx, const float* const* L, int T, int h, int w,
                                       int ldl, const lp_spectrum* const* spectra, float* out,
                                       int ldo, lp_outmode mode, lp_precision prec, void* stream)
{
    if (!L || T < 1) return lp_fail(LP_ERR_INVALID, "lp_map_multiclass: need T >= 1 maps");
    if (T > kMaxSpectraPerLaunch)
        return lp_fail(LP_ERR_INVALID, "lp_map_multiclass: at most %d classes", kMaxSpectraPerLaunch);
    for (int t = 0; t < T; ++t)
        if (!L[t]) return lp_fail(LP_ERR_INVALID, "lp_map_multiclass: L[%d] is NULL", t);
    MapDims d;
    if (prec != LP_PREC_FP32)
        return lp_fail(LP_ERR_UNSUPPORTED, "lp_map_multiclass: only the FP32 path is built for several classes");
    lp_status st = lp_validate_map(ctx, L[0], h, w, ldl, spectra, T, out, ldo, mode, prec, &d);
    if (st != LP_OK) return st;
    if (mode == LP_OUT_SAME) {
        // the crop offset is zero for every spectrum; FULL needs equal PSF sizes (checked)
    }
    DeviceGuard dg(ctx->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const lp_spectrum* s0 = spectra[0];
    const PlanRec *py, *px;
    if ((st = lp_get_plan(ctx, s0->ny, &py)) != LP_OK) return st;
    if ((st = lp_get_plan(ctx, s0->nx, &px)) != LP_OK) return st;
    const size_t tbytes = 8ull * (size_t)d.ncolsT * d.ldT;
    const size_t ubytes = 8ull * (size_t)d.ncolsU * d.ldU;
    void* ws = nullptr;
    if ((st = lp_get_workspace(ctx, s, (size_t)T * tbytes + ubytes + lp_park_bytes(d) + 512, &ws)) != LP_OK)
        return st;
    float2* Tb = static_cast<float2*>(ws);
    float2* U = Tb + (size_t)T * d.ncolsT * d.ldT;
    float2* accb = park_of(d, U, 1);
    const int npairs = (int)(d.ldT / 2);
    if ((st = lp_wait_spectra_built(spectra, T, s)) != LP_OK) return st;
    for (int t = 0; t < T; ++t) {
        P1Args a1;
        a1.L = L[t];
        a1.ldl = ldl;
        a1.H = h;
        a1.W = w;
        a1.Wst = (w + 3) / 4 * 4;
        a1.vec16 = ((reinterpret_cast<uintptr_t>(L[t]) & 15) == 0 && ldl % 4 == 0 && w % 4 == 0) ? 1 : 0;
        a1.T = Tb + (size_t)t * d.ncolsT * d.ldT;
        a1.ldT = d.ldT;
        a1.pair0 = 0;
        a1.npairs = npairs;
        a1.ncols = d.ncols;
        a1.tw = px->fwd;
        a1.err = ctx->d_err;
        a1.t_elems = t_extent(ctx, d);
        CUDA_TRY(px->k->p1(a1, s));
    }
    // the real-spectrum kernel needs every class's spectrum real
    bool all_real = true;
    for (int t = 0; t < T; ++t) all_real = all_real && spectra[t]->is_real;
    if (!all_real)
        for (int t = 0; t < T; ++t)
            if (spectra[t]->is_real)
                return lp_fail(LP_ERR_UNSUPPORTED,
                               "lp_map_multiclass: mixing real and complex spectra is not supported");
    P2MArgs a2;
    for (int i = 0; i < kMaxSpectraPerLaunch; ++i) {
        a2.T[i] = i < T ? Tb + (size_t)i * d.ncolsT * d.ldT : nullptr;
        a2.K[i] = i < T ? spectra[i]->data : nullptr;
    }
    a2.ldT = d.ldT;
    a2.H = h;
    a2.ldK = s0->ldK;
    a2.nclass = T;
    a2.U = U;
    a2.ldU = d.ldU;
    a2.r0 = d.r0;
    a2.Hout = d.Hout;
    a2.HoutPad = (int)d.ldU;
    a2.ncols = d.ncols;
    a2.twf = py->fwd;
    a2.twi = py->rev;
    a2.acc = accb;
    a2.err = ctx->d_err;
    a2.t_elems = t_extent(ctx, d);
    a2.k_elems = k_extent(spectra[0]);
    for (int t = 1; t < T; ++t) a2.k_elems = std::min(a2.k_elems, k_extent(spectra[t]));
    a2.u_elems = (long long)d.ncolsU * d.ldU;
    a2.acc_elems = (long long)d.ncols * d.ny;
    {
        const cudaError_t e = py->k->p2m(a2, all_real, s);
        if (e != cudaSuccess) return lp_fail(LP_ERR_CUDA, "lp_map_multiclass: %s", cudaGetErrorString(e));
    }
    P3Args a3;
    a3.U = U;
    a3.ldU = d.ldU;
    a3.specU = 0;
    a3.Hout = d.Hout;
    a3.pair0 = 0;
    a3.npairs = (int)(d.ldU / 2);
    for (int i = 0; i < kMaxSpectraPerLaunch; ++i) a3.out[i] = i == 0 ? out : nullptr;
    a3.ldo = ldo;
    a3.c0 = d.c0;
    a3.Wout = d.Wout;
    a3.ncols = d.ncols;
    a3.tw = px->rev;
    a3.err = ctx->d_err;
    a3.u_elems = (long long)d.ncolsU * d.ldU;
    CUDA_TRY(px->k->p3(a3, 1, s));
    lp_note_spectra_used(ctx, spectra, T, s);
    return LP_OK;
}

// ---------------------------------------------------------------------------
// pass timing
// ---------------------------------------------------------------------------
static cudaEvent_t pool_event(lp_ctx* ctx)
{
    if (!ctx->tim_pool.empty()) {
        cudaEvent_t e = ctx->tim_pool.back();
        ctx->tim_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

int lp_pass_begin(lp_ctx* ctx, int pass, cudaStream_t s)
{
    std::lock_guard<std::mutex> g(ctx->tim_mu);
    if (!ctx->timing) return -1;
    PassEvent pe{pass, pool_event(ctx), pool_event(ctx)};
    if (!pe.start || !pe.stop) return -1;
    cudaEventRecord(pe.start, s);
    ctx->tim_pending.push_back(pe);
    return (int)ctx->tim_pending.size() - 1;
}

void lp_pass_end(lp_ctx* ctx, int token, cudaStream_t s)
{
    if (token < 0) return;
    std::lock_guard<std::mutex> g(ctx->tim_mu);
    if (token < (int)ctx->tim_pending.size()) cudaEventRecord(ctx->tim_pending[token].stop, s);
}

extern "C" lp_status lp_set_pass_timing(lp_ctx* ctx, int enable)
{
    if (!ctx) return lp_fail(LP_ERR_INVALID, "lp_set_pass_timing: NULL context");
    std::lock_guard<std::mutex> g(ctx->tim_mu);
    ctx->timing = enable != 0;
    return LP_OK;
}

extern "C" lp_status lp_get_pass_timing(lp_ctx* ctx, double* ms, int* launches)
{
    if (!ctx || !ms || !launches) return lp_fail(LP_ERR_INVALID, "lp_get_pass_timing: NULL argument");
    DeviceGuard dg(ctx->device);
    std::lock_guard<std::mutex> g(ctx->tim_mu);
    for (int i = 0; i < 3; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
    }
    for (auto& pe : ctx->tim_pending) {
        CUDA_TRY(cudaEventSynchronize(pe.stop));
        float t = 0.f;
        CUDA_TRY(cudaEventElapsedTime(&t, pe.start, pe.stop));
        if (pe.pass >= 0 && pe.pass < 3) {
            ms[pe.pass] += t;
            launches[pe.pass] += 1;
        }
        ctx->tim_pool.push_back(pe.start);
        ctx->tim_pool.push_back(pe.stop);
    }
    ctx->tim_pending.clear();
    return LP_OK;
}
