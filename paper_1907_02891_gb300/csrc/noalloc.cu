// lp_map_noalloc: the map with its scratch in a static device array.
//
// lp_map keeps its intermediate spectra (T and U) in a per-stream workspace
// that the context allocates with cudaMalloc the first time a size needs
// it.  Some callers cannot have that happen while they run: a host
// framework that owns all device memory through its own pool and budget
// (a cudaMalloc behind its back breaks its accounting), or a latency-bound
// loop where the allocation and the device synchronisation it implies are
// not acceptable.  This entry point allocates nothing: the scratch lives in
// the file-scope array below, which every GPU that loads this code holds
// until the process exits.
//
// Set-up: the first call on a device (with that device current) asks the
// runtime for the array's device address with cudaGetSymbolAddress and
// caches it; make that first call before any stream capture.  The host-side
// name of the array is only a stand-in for it and is never passed to a
// kernel.
//
// Sharing: every call on a device uses the same array and leaves its
// contents behind.  The kernels overwrite every scratch element they later
// read (the row-transform pass writes all of T, the column pass all kept
// rows of U plus the padding row, which it zeroes), so nothing needs
// clearing between calls.  Calls whose work overlaps on the GPU (other
// streams, other threads) race on the array: serialise them.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/lp.h"
#include "lp_runtime.h"

namespace {

constexpr size_t kScratchBytes = LP_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

lp_status scratch_address(int device, void** out)
{
    std::lock_guard<std::mutex> g(g_mu);
    if (device < 0 || device >= kMaxDevices)
        return lp_fail(LP_ERR_INVALID, "lp_map_noalloc: device %d out of range", device);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess || !p)
            return lp_fail(LP_ERR_CUDA, "lp_map_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return LP_OK;
}

struct CurrentDevice {
    int prev = -1;
    bool ok = true;
    explicit CurrentDevice(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~CurrentDevice()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

bool plan_cached(lp_ctx* ctx, int n)
{
    std::lock_guard<std::mutex> g(ctx->plan_mu);
    return ctx->plans.find(n) != ctx->plans.end();
}

}  // namespace

extern "C" size_t lp_map_noalloc_scratch_bytes(void) { return kScratchBytes; }

extern "C" lp_status lp_map_noalloc(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                                    const lp_spectrum* const* spectra, int n, float* const* out,
                                    int ldo, lp_outmode mode, lp_precision prec, void* stream)
{
    MapDims d;
    lp_status st = lp_validate_map(ctx, L, h, w, ldl, spectra, n, out, ldo, mode, prec, &d);
    if (st != LP_OK) return st;
    for (int k = 0; k < n; ++k) {
        if (!out[k]) return lp_fail(LP_ERR_INVALID, "lp_map_noalloc: out[%d] is NULL", k);
        const char* o0 = reinterpret_cast<const char*>(out[k]);
        const char* o1 = o0 + 4ull * ((size_t)(d.Hout - 1) * ldo + d.Wout);
        const char* l0 = reinterpret_cast<const char*>(L);
        const char* l1 = l0 + 4ull * ((size_t)(h - 1) * ldl + w);
        if (o0 < l1 && l0 < o1) return lp_fail(LP_ERR_INVALID, "lp_map_noalloc: out[%d] overlaps L", k);
    }
    const lp_spectrum* s0 = spectra[0];
    const size_t need = lp_map_workspace_bytes(h, w, s0->ny, s0->nx, s0->hk, s0->wk, n, mode);
    if (need > kScratchBytes)
        return lp_fail(LP_ERR_INVALID,
                       "lp_map_noalloc: this map needs %zu bytes of scratch; the static scratch "
                       "holds %zu (use lp_map, or a smaller map / fewer spectra)",
                       need, kScratchBytes);
    // plans (twiddle tables) are built when the spectra are created; a
    // missing one would have to be allocated, so refuse instead
    if (!plan_cached(ctx, s0->ny) || !plan_cached(ctx, s0->nx))
        return lp_fail(LP_ERR_INVALID, "lp_map_noalloc: no cached plan for %d x %d", s0->ny, s0->nx);
    {
        std::lock_guard<std::mutex> g(ctx->tim_mu);
        if (ctx->timing)
            return lp_fail(LP_ERR_INVALID, "lp_map_noalloc: switch pass timing off first (it creates events)");
    }
    CurrentDevice cd(ctx->device);
    if (!cd.ok) return lp_fail(LP_ERR_CUDA, "lp_map_noalloc: cudaSetDevice(%d) failed", ctx->device);
    void* scratch = nullptr;
    if ((st = scratch_address(ctx->device, &scratch)) != LP_OK) return st;
    return lp_launch_map(ctx, L, h, w, ldl, spectra, n, out, ldo, d, scratch,
                         static_cast<cudaStream_t>(stream));
}
