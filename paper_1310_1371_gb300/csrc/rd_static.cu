// rd_static.cu -- rd_ridges_static: the directed-ridge stages (smoothing,
// exact Hessian, ridge mask, direction refinement) of one frame, with no
// device allocation.
//
// Who needs it: callers that cannot allocate device memory where they call
// the detector.  Acquisition loops that forbid cudaMalloc on the per-frame
// path (it can synchronise the whole device and its latency is unbounded);
// plug-ins whose host application owns every device allocation through its
// own pool; processes whose device memory another framework has already
// reserved.  rd_create allocates a context's workspaces; this entry point
// needs none: its scratch memory is one fixed array in this file, which
// every GPU that loads the library holds until the process exits.
#include "rd_internal.cuh"
#include "rd_abi_guard.h"

#include <cuda.h>
#include <cstddef>
#include <mutex>
#include <string>

namespace rd {

// The most stencil tiles a frame within the limits can have (each side in
// [12, 65535], at most RD_STATIC_MAX_PIXELS pixels): 2048, at 12 x 65535 (one
// row of tiles).
constexpr long long static_tiles_bound() {
  long long best = 0;
  for (long long h = 12; h <= 65535; ++h) {
    long long w = RD_STATIC_MAX_PIXELS / h;
    if (w > 65535) w = 65535;
    if (w < 12) break;
    const long long t = ((h + ST_TH - 1) / ST_TH) * ((w + ST_TW - 1) / ST_TW);
    if (t > best) best = t;
  }
  return best;
}
constexpr int STATIC_MAX_TILES = 2048;
static_assert(static_tiles_bound() <= STATIC_MAX_TILES, "stencil tile index too small for the frame limits");

// Scratch of one call: K1's counters, its per-tile record index, the exact
// Hessians it writes beside the caller's ridge list, and the vote-rounding
// margins K2 writes beside the caller's directions.  About 8.4 MB.
struct StaticScratch {
  DevStats stats;
  int tile_off[STATIC_MAX_TILES];
  int tile_cnt[STATIC_MAX_TILES];
  long long hess[3 * (size_t)RD_STATIC_MAX_RIDGE];
  float2 kvote[RD_STATIC_MAX_RIDGE];
};

static __device__ __align__(256) StaticScratch g_rd_static_scratch;

namespace {
constexpr int MAX_DEVICES = 64;

struct DeviceSetup {
  StaticScratch* scratch;      // device address of g_rd_static_scratch in the context below
  unsigned long long ctx_id;   // unique id of the CUDA context the address was looked up in
  int n_sm;
};

std::mutex g_setup_mutex;
DeviceSetup g_setup[MAX_DEVICES] = {};
thread_local std::string g_static_error;

// Driver entry points for the current context's identity, fetched through
// the runtime so that the library does not link the driver library itself.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

rd_status fail_static(rd_status s, const std::string& m) {
  g_static_error = m;
  return s;
}

rd_status fail_cuda(const char* what, cudaError_t e) {
  return fail_static(RD_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Unique id of the calling thread's current CUDA context, 0 if none is
// current yet.  Caller holds g_setup_mutex.
rd_status current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1);
    if (e == cudaSuccess)
      e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2);
    if (e != cudaSuccess) return fail_cuda("cudaGetDriverEntryPointByVersion", e);
    if (q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess || !f1 || !f2)
      return fail_static(RD_E_CUDA, "the driver has no cuCtxGetCurrent / cuCtxGetId");
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return fail_static(RD_E_CUDA, "cuCtxGetCurrent failed");
  *id = 0;
  if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return fail_static(RD_E_CUDA, "cuCtxGetId failed");
  return RD_OK;
}

// Set-up for the current device and context: the scratch array's device
// address (its host-side name is only a stand-in for the symbol) and the SM
// count that sizes the refinement grid.  The address belongs to the context
// it was looked up in, so it is cached per device together with that
// context's unique id, and looked up again when another context is current
// (a context rebuilt after cudaDeviceReset, or one the caller created with
// the driver API).  A look-up loads the library's module into the context,
// so the first call in each context must not be inside a stream capture.
rd_status setup_current_device(DeviceSetup* out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_cuda("cudaGetDevice", e);
  if (dev < 0 || dev >= MAX_DEVICES) return fail_static(RD_E_INVAL, "device index above 63");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  unsigned long long id = 0;
  rd_status st = current_context_id(&id);
  if (st != RD_OK) return st;
  DeviceSetup& s = g_setup[dev];
  if (!s.scratch || id == 0 || s.ctx_id != id) {
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return fail_cuda("cudaDeviceGetAttribute", e);
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_rd_static_scratch);  // makes the device's primary context current
    if (e != cudaSuccess) return fail_cuda("cudaGetSymbolAddress", e);
    if (!p) return fail_static(RD_E_CUDA, "cudaGetSymbolAddress returned NULL");
    if (id == 0) {  // no context was current before the look-up: take the one it used
      st = current_context_id(&id);
      if (st != RD_OK) return st;
    }
    s.n_sm = n_sm > 0 ? n_sm : 1;
    s.scratch = static_cast<StaticScratch*>(p);
    s.ctx_id = id;
  }
  *out = s;
  return RD_OK;
}
}  // namespace

}  // namespace rd

using namespace rd;

extern "C" const char* rd_static_last_error(void) { return g_static_error.c_str(); }

extern "C" rd_status rd_ridges_static(const rd_params* p, const void* frame_dev, int H, int W, int dtype,
                                      void* stream, uint32_t* xy_dev, float* dir_dev, int cap,
                                      int* count_dev) {
  return rd_abi::guard(&g_static_error, [&]() -> rd_status {
    if (!p || !frame_dev || !xy_dev || !dir_dev || !count_dev) return fail_static(RD_E_INVAL, "NULL argument");
    if (!(p->sigma > 0.0f && p->sigma <= 4.0f)) return fail_static(RD_E_INVAL, "sigma must be in (0, 4]");
    if (!(p->ridge_thresh <= 0.0f)) return fail_static(RD_E_INVAL, "ridge_thresh must be <= 0");
    if (dtype != RD_U8 && dtype != RD_U16) return fail_static(RD_E_INVAL, "dtype must be RD_U8 or RD_U16");
    GaussTaps taps;
    taps.R = (rd_gaussian_taps(p->sigma, taps.q, 2 * MAX_RG + 1) - 1) / 2;
    if (taps.R < 1) return fail_static(RD_E_INVAL, "sigma gives no Gaussian taps");
    if (H < taps.R + 4 || W < taps.R + 4 || H < 12 || W < 12 || H > 65535 || W > 65535)
      return fail_static(RD_E_INVAL, "frame size must be in [max(12, ceil(4 sigma) + 4), 65535]");
    if ((long long)H * W > RD_STATIC_MAX_PIXELS)
      return fail_static(RD_E_INVAL, "frame has more than RD_STATIC_MAX_PIXELS (1048576) pixels");
    const int n_stx = (W + ST_TW - 1) / ST_TW, n_sty = (H + ST_TH - 1) / ST_TH;
    if ((long long)n_stx * n_sty > STATIC_MAX_TILES)
      return fail_static(RD_E_INVAL, "frame has more stencil tiles than the static scratch holds");
    if (cap < 0 || cap > RD_STATIC_MAX_RIDGE)
      return fail_static(RD_E_INVAL, "cap must be in [0, RD_STATIC_MAX_RIDGE] (262144)");
    if (((uintptr_t)dir_dev & 15) != 0) return fail_static(RD_E_INVAL, "dir_dev must be 16-byte aligned");
    if (((uintptr_t)xy_dev & 3) != 0) return fail_static(RD_E_INVAL, "xy_dev must be 4-byte aligned");
    if (((uintptr_t)count_dev & 3) != 0) return fail_static(RD_E_INVAL, "count_dev must be 4-byte aligned");
    if (dtype == RD_U16 && ((uintptr_t)frame_dev & 1) != 0)
      return fail_static(RD_E_INVAL, "frame_dev must be 2-byte aligned for RD_U16");

    DeviceSetup dev;
    rd_status s = setup_current_device(&dev);
    if (s != RD_OK) return s;
    StaticScratch* sc = dev.scratch;
    cudaStream_t st = (cudaStream_t)stream;

    // The array keeps the previous call's contents.  The counters must start at
    // zero; the tile index, Hessians and margins are written before they are
    // read.
    cudaError_t e = cudaMemsetAsync(count_dev, 0, sizeof(int), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(&sc->stats, 0, sizeof(DevStats), st);
    if (e != cudaSuccess) return fail_cuda("cudaMemsetAsync", e);

    long long S = 0;
    for (int i = 0; i <= 2 * taps.R; ++i) S += taps.q[i];
    StencilArgs a{};
    a.edge = 0;
    a.frames = frame_dev;
    a.n = 1;
    a.H = H;
    a.W = W;
    a.taps = taps;
    a.tau = p->ridge_thresh;
    a.tau64 = (double)p->ridge_thresh;
    a.D64 = (double)(64LL * S * S);
    a.invD = (float)(1.0 / a.D64);
    a.rl.xy = xy_dev;
    a.rl.dir = reinterpret_cast<float4*>(dir_dev);
    a.rl.kvote = sc->kvote;
    a.rl.hess = sc->hess;
    a.rl.count = count_dev;
    a.rl.tile_off = sc->tile_off;
    a.rl.tile_cnt = sc->tile_cnt;
    a.rl.cap = cap;
    a.rl.n_stx = n_stx;
    a.rl.n_sty = n_sty;
    a.stats = &sc->stats;
    e = launch_stencil(a, dtype, st);
    if (e != cudaSuccess) return fail_cuda("stencil launch", e);
    e = launch_refine(a.rl, 1, dev.n_sm, st);
    if (e != cudaSuccess) return fail_cuda("refine launch", e);
    return RD_OK;
  });
}
