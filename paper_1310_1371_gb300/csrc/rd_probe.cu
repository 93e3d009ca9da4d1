// rd_probe.cu -- a measured peak for the roofline of the voting stage: the
// rate at which this GPU executes shared-memory atomic adds, the operation
// that accumulates votes (Results, "Directed ridge detection & votes
// collection"; Detailed algorithm step 4, level population).
//
// Each CTA owns a 32 KB array of u32 counters in shared memory (the size of
// one level of a 128 x 128 accumulator tile of packed u16 counts) and adds to
// it in a fixed, unrolled loop.  Three address patterns:
//   0  conflict-free: the 32 lanes of a warp hit 32 distinct banks (u32 adds);
//   1  packed u16 pairs: lanes 2j and 2j + 1 add 1 and 2^16 to the same word,
//      as two votes for horizontally adjacent voxels do;
//   2  random: every lane adds 1 or 2^16 to a pseudo-random word of the
//      array, the address distribution of a warp's votes (one ridge pixel per
//      lane, positions spread over the tile).
// Addresses are computed before the timed loop and masked into the array.
#include "rd_internal.cuh"

#include <string>

namespace rd {

constexpr int PROBE_WORDS = 8192;  // 32 KB
constexpr int PROBE_THREADS = 256;
constexpr int PROBE_UNROLL = 8;

__device__ __forceinline__ uint32_t probe_hash(uint32_t x) {
  // integer mixing (xorshift-multiply rounds)
  x ^= x >> 16;
  x *= 0x7feb352du;
  x ^= x >> 15;
  x *= 0x846ca68bu;
  x ^= x >> 16;
  return x;
}

template <int PAT>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_smem_atomics(int iters, uint32_t seed, unsigned* sink) {
  __shared__ uint32_t s[PROBE_WORDS];
  for (int i = threadIdx.x; i < PROBE_WORDS; i += PROBE_THREADS) s[i] = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t addr[PROBE_UNROLL], val[PROBE_UNROLL];
#pragma unroll
  for (int k = 0; k < PROBE_UNROLL; ++k) {
    if (PAT == 0) {
      addr[k] = (uint32_t)(warp * 32 + lane + k * PROBE_THREADS) & (PROBE_WORDS - 1);
      val[k] = 1u;
    } else if (PAT == 1) {
      addr[k] = (uint32_t)(warp * 16 + (lane >> 1) + k * (PROBE_THREADS / 2)) & (PROBE_WORDS - 1);
      val[k] = (lane & 1) ? 65536u : 1u;
    } else {
      const uint32_t h = probe_hash(seed ^ probe_hash((blockIdx.x * PROBE_THREADS + threadIdx.x) * 8u + k));
      addr[k] = h & (PROBE_WORDS - 1);
      val[k] = (h >> 13) & 1u ? 65536u : 1u;
    }
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int k = 0; k < PROBE_UNROLL; ++k) atomicAdd(&s[addr[k]], val[k]);
  }
  __syncthreads();
  // keep the counts observable: fold them into one global word per CTA
  uint32_t t = 0;
  for (int i = threadIdx.x; i < PROBE_WORDS; i += PROBE_THREADS) t += s[i];
  t = __reduce_add_sync(0xffffffffu, t);
  if (lane == 0) atomicAdd(sink, t);
}

}  // namespace rd

using namespace rd;

static thread_local std::string g_probe_error;

extern "C" const char* rd_probe_last_error(void) { return g_probe_error.c_str(); }

extern "C" rd_status rd_probe_smem_atomics(int pattern, int ctas_per_sm, int iters, void* stream,
                                           double* atomics_per_s, float* ms) {
  if (!atomics_per_s || pattern < 0 || pattern > 2 || ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 ||
      iters > (1 << 20)) {
    g_probe_error = "pattern must be 0-2, ctas_per_sm 1-8, iters 1-2^20, atomics_per_s non-NULL";
    return RD_E_INVAL;
  }
  auto cuda_fail = [](const char* what, cudaError_t e) {
    g_probe_error = std::string(what) + ": " + cudaGetErrorString(e);
    return RD_E_CUDA;
  };
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_fail("device query", e);
  cudaStream_t st = (cudaStream_t)stream;
  unsigned* sink = nullptr;
  e = cudaMalloc(&sink, sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail("cudaMalloc", e);
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  const int grid = n_sm * ctas_per_sm;
  auto launch = [&](int it) {
    if (pattern == 0) k_probe_smem_atomics<0><<<grid, PROBE_THREADS, 0, st>>>(it, 0x2545f491u, sink);
    else if (pattern == 1) k_probe_smem_atomics<1><<<grid, PROBE_THREADS, 0, st>>>(it, 0x2545f491u, sink);
    else k_probe_smem_atomics<2><<<grid, PROBE_THREADS, 0, st>>>(it, 0x2545f491u, sink);
    return cudaGetLastError();
  };
  float t = 0.0f;
  if (e == cudaSuccess) e = launch(iters);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(ev[0], st);
  if (e == cudaSuccess) e = launch(iters);
  if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
  for (auto& v : ev)
    if (v) cudaEventDestroy(v);
  cudaFree(sink);
  if (e != cudaSuccess) return cuda_fail("probe", e);
  const double n = (double)grid * PROBE_THREADS * PROBE_UNROLL * (double)iters;
  *atomics_per_s = n / ((double)t * 1e-3);
  if (ms) *ms = t;
  return RD_OK;
}
