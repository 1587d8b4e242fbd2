// Host-side state of a context (shared by api.cu and serve.cpp).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <map>
#include <memory>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/lp.h"
#include "lp_internal.h"

struct SpecKey {
    unsigned long long fp;  // order-independent fingerprint of the PSF values
    int hk, wk, ny, nx, prec;
    int salt;  // tells apart different PSFs whose fingerprints collide
    bool operator<(const SpecKey& o) const
    {
        return std::tie(fp, hk, wk, ny, nx, prec, salt) < std::tie(o.fp, o.hk, o.wk, o.ny, o.nx, o.prec, o.salt);
    }
    bool same_request(const SpecKey& o) const
    {
        return fp == o.fp && hk == o.hk && wk == o.wk && ny == o.ny && nx == o.nx && prec == o.prec;
    }
};

struct PlanRec {
    const lpk::SizeKernels* k = nullptr;
    float2* tw = nullptr;  // device twiddle tables (forward chain, then reversed chain)
    size_t bytes = 0;
    lpk::TwChain fwd{}, rev{};
    // tables of the tensor-core column pass (split-BF16 DFT matrices, then
    // twiddle step factors; same block as tw; null where the length has no
    // such pass)
    const void* tc_tables = nullptr;
};

struct Workspace {
    cudaStream_t stream;
    void* ptr;
    size_t bytes;
};

struct MapDims {
    int ncols;          // Nx/2 + 1
    long long ncolsT;   // columns allocated for T (ncols rounded up to its column blocks)
    long long ncolsU;   // columns allocated per spectrum for U (likewise)
    long long ldT, ldU; // leading dimensions of T and U (complex elements, even)
    int Hout, Wout;     // output size
    int r0, c0;         // first kept row / column of the circular result
    int prec;           // lp_precision of the column pass
    int ny;             // padded column length
    int batch;          // several FP32 spectra share one forward column transform
};

struct ServeState;

struct PassEvent {
    int pass;
    cudaEvent_t start, stop;
};

struct lp_spectrum {
    lp_ctx* ctx = nullptr;
    SpecKey key{};
    int ny = 0, nx = 0, hk = 0, wk = 0, is_real = 0;
    lp_precision prec = LP_PREC_FP32;
    long long ldK = 0;  // elements per stored column-frequency row
    size_t bytes = 0;
    int refcount = 0;
    void* data = nullptr;
    cudaEvent_t ready = nullptr;  // recorded after the build on the building stream
    std::atomic<bool> built{false};  // `ready` has been seen complete
    // device copy of K (hk x wk FP64): a cache hit is confirmed by comparing
    // the requested PSF with it value by value
    double* kcopy = nullptr;
    size_t kbytes = 0;
    // Last use per stream, for stream-ordered release: every map call
    // re-records the event of its stream's slot at its end.  Streams beyond
    // the slots set `use_overflow`, and the release then waits for the device.
    static constexpr int kUseSlots = 8;
    cudaStream_t use_stream[kUseSlots] = {};
    cudaEvent_t use_event[kUseSlots] = {};
    int nuse = 0;
    bool use_overflow = false;
};

struct lp_ctx {
    int device = 0;
    int sms = 0;  // multiprocessors of the device (0: not looked up yet)
    size_t budget = 0, used = 0;
    std::mutex mem_mu, plan_mu, spec_mu, ws_mu;
    std::map<int, std::unique_ptr<PlanRec>> plans;
    std::map<SpecKey, lp_spectrum*> spectra;
    // released spectra whose last uses may still be running: freed once
    // their build and use events have completed
    std::vector<lp_spectrum*> released;
    std::vector<Workspace> ws;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    int* d_err = nullptr;  // sticky device status word
    std::atomic<int> test_hook{0};  // lp_set_test_hook bits (read by the serving thread too)
    ServeState* serve = nullptr;
    // pass timing
    std::mutex tim_mu;
    bool timing = false;
    std::vector<PassEvent> tim_pending;
    std::vector<cudaEvent_t> tim_pool;
    // pipelined host-buffer map
    std::mutex host_mu;
    cudaStream_t hs_in = nullptr, hs_out = nullptr, hs_comp = nullptr;
    std::vector<cudaEvent_t> hs_events;
    cudaEvent_t hs_lfree[2] = {nullptr, nullptr};  // row pass done with input staging b
    bool hs_lfree_valid[2] = {false, false};
    int hs_lbuf = 0;  // input staging buffer of the next host map
    cudaEvent_t hs_ofree[2] = {nullptr, nullptr};  // download from output staging b done
    bool hs_ofree_valid[2] = {false, false};
    int hs_obuf = 0;  // output staging buffer of the next host map
};

lp_status lp_fail(lp_status st, const char* fmt, ...);
lp_status lp_ctx_alloc(lp_ctx* ctx, size_t bytes, void** p);
void lp_ctx_free(lp_ctx* ctx, void* p, size_t bytes);
lp_status lp_get_plan(lp_ctx* ctx, int N, const PlanRec** out);
lp_status lp_get_workspace(lp_ctx* ctx, cudaStream_t s, size_t bytes, void** out);
// true while stream s is being captured into a CUDA graph
bool lp_stream_capturing(cudaStream_t s);
lp_status lp_validate_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                          const lp_spectrum* const* spectra, int n, const void* out, int ldo,
                          lp_outmode mode, lp_precision prec, MapDims* d);
// bytes of one map's workspace: T, then U for up to kMaxSpectraPerLaunch
// spectra (the spectra of one launch), + alignment slack
size_t lp_workspace_bytes(const MapDims& d, int n);
// parked forward column spectra of the batched column pass: Ny complex per column
size_t lp_park_bytes(const MapDims& d);
lp_status lp_launch_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                        const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                        const MapDims& d, void* ws, cudaStream_t st);
void lp_serve_shutdown(lp_ctx* ctx);
// Map calls wait, in stream order, for the builds of their spectra that are
// not yet known to be complete (no wait once a build has been seen done).
lp_status lp_wait_spectra_built(const lp_spectrum* const* spectra, int n, cudaStream_t st);
// Records the end of a map call on stream st as the last use of each spectrum.
void lp_note_spectra_used(lp_ctx* ctx, const lp_spectrum* const* spectra, int n, cudaStream_t st);
// Reference counting shared by lp_spectrum_release and the request scheduler
// (which holds one reference per queued or running request).
void lp_spectrum_ref(lp_ctx* ctx, const lp_spectrum* s);
lp_status lp_spectrum_unref(lp_ctx* ctx, const lp_spectrum* s);
// Frees released spectra whose last uses are complete; wait = block for them.
void lp_reap_released(lp_ctx* ctx, bool wait);
// records the start of pass `pass` on stream s when timing is on; returns a
// token for lp_pass_end (-1 when off)
int lp_pass_begin(lp_ctx* ctx, int pass, cudaStream_t s);
void lp_pass_end(lp_ctx* ctx, int token, cudaStream_t s);
