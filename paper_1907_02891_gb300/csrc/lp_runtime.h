// Host-side state of a context (shared by api.cu and serve.cpp).
#pragma once

#include <cuda_runtime.h>

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
    bool operator<(const SpecKey& o) const
    {
        return std::tie(fp, hk, wk, ny, nx, prec) < std::tie(o.fp, o.hk, o.wk, o.ny, o.nx, o.prec);
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
};

struct lp_ctx {
    int device = 0;
    size_t budget = 0, used = 0;
    std::mutex mem_mu, plan_mu, spec_mu, ws_mu;
    std::map<int, std::unique_ptr<PlanRec>> plans;
    std::map<SpecKey, lp_spectrum*> spectra;
    std::vector<Workspace> ws;
    void* staging = nullptr;
    size_t staging_bytes = 0;
    int* d_err = nullptr;  // sticky device status word
    int test_hook = 0;     // lp_set_test_hook
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
    cudaEvent_t hs_lfree = nullptr;  // previous host map's row pass done with the staging map
    bool hs_lfree_valid = false;
    cudaEvent_t hs_ofree[2] = {nullptr, nullptr};  // download from output staging b done
    bool hs_ofree_valid[2] = {false, false};
    int hs_obuf = 0;  // output staging buffer of the next host map
};

lp_status lp_fail(lp_status st, const char* fmt, ...);
lp_status lp_ctx_alloc(lp_ctx* ctx, size_t bytes, void** p);
void lp_ctx_free(lp_ctx* ctx, void* p, size_t bytes);
lp_status lp_get_plan(lp_ctx* ctx, int N, const PlanRec** out);
lp_status lp_get_workspace(lp_ctx* ctx, cudaStream_t s, size_t bytes, void** out);
lp_status lp_validate_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                          const lp_spectrum* const* spectra, int n, const void* out, int ldo,
                          lp_outmode mode, lp_precision prec, MapDims* d);
// bytes of one map's workspace: T, then U for up to kMaxSpectraPerLaunch
// spectra (the spectra of one launch), + alignment slack
size_t lp_workspace_bytes(const MapDims& d, int n);
lp_status lp_launch_map(lp_ctx* ctx, const float* L, int h, int w, int ldl,
                        const lp_spectrum* const* spectra, int n, float* const* out, int ldo,
                        const MapDims& d, void* ws, cudaStream_t st);
void lp_serve_shutdown(lp_ctx* ctx);
// records the start of pass `pass` on stream s when timing is on; returns a
// token for lp_pass_end (-1 when off)
int lp_pass_begin(lp_ctx* ctx, int pass, cudaStream_t s);
void lp_pass_end(lp_ctx* ctx, int token, cudaStream_t s);
