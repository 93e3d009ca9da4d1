// k_fit.cu -- per-frame ordering of the integer peaks and K5: annulus
// classification of ridge pixels and a circle fit per peak.
//
// Method: Results ("Ridge points classification & sub-pixel accuracy": an
// annulus mask per peak, a best-fitting circle through the ridge pixels it
// covers, non-exclusive membership); Detailed algorithm step 5.  The fit is
// the algebraic least-squares circle (Kasa): minimise
// sum (u^2 + v^2 + D u + E v + F)^2 over the offsets (u, v) = p - c.
#include "rd_internal.cuh"

namespace rd {

constexpr int SORT_THREADS = 1024;

// One CTA per frame: bitonic sort of the frame's peaks by (r, y, x).
__global__ void __launch_bounds__(SORT_THREADS) k_sort_peaks(int4* peaks, const int* peak_count, int cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  unsigned long long* key = reinterpret_cast<unsigned long long*>(smem);
  uint32_t* val = reinterpret_cast<uint32_t*>(key + cap);
  const int f = blockIdx.x;
  const int n = min(peak_count[f], cap);
  if (n <= 1) return;
  int np = 1;
  while (np < n) np <<= 1;
  int4* P = peaks + (size_t)f * cap;
  for (int i = threadIdx.x; i < np; i += SORT_THREADS) {
    if (i < n) {
      int4 p = P[i];
      key[i] = ((unsigned long long)p.z << 40) | ((unsigned long long)p.y << 20) | (unsigned long long)p.x;
      val[i] = (uint32_t)p.w;
    } else {
      key[i] = ~0ULL;
      val[i] = 0;
    }
  }
  __syncthreads();
  for (int k = 2; k <= np; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np; i += SORT_THREADS) {
        int l = i ^ j;
        if (l > i) {
          bool up = (i & k) == 0;
          unsigned long long a = key[i], b = key[l];
          if ((a > b) == up) {
            key[i] = b;
            key[l] = a;
            uint32_t t = val[i];
            val[i] = val[l];
            val[l] = t;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < n; i += SORT_THREADS) {
    unsigned long long k = key[i];
    P[i] = make_int4((int)(k & 0xfffffULL), (int)((k >> 20) & 0xfffffULL), (int)(k >> 40), (int)val[i]);
  }
}

// Single CTA: counts (true peak counts) and their exclusive prefix sum.
__global__ void k_ring_offsets(const int* peak_count, int n_frames, int* counts, int* offsets) {
  __shared__ int s[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < n_frames; base += 1024) {
    int i = base + threadIdx.x;
    int v = i < n_frames ? peak_count[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    if (i < n_frames) {
      counts[i] = v;
      offsets[i] = s[threadIdx.x] - v + carry;
    }
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
}


__device__ __forceinline__ double i128_to_double(__int128 x) {
  bool neg = x < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-x) : (unsigned __int128)x;
  double hi = (double)(unsigned long long)(u >> 64), lo = (double)(unsigned long long)u;
  double d = hi * 18446744073709551616.0 + lo;
  return neg ? -d : d;
}

__device__ __forceinline__ __int128 det3(const long long m[3][3]) {
  __int128 a = (__int128)m[1][1] * m[2][2] - (__int128)m[1][2] * m[2][1];
  __int128 b = (__int128)m[1][0] * m[2][2] - (__int128)m[1][2] * m[2][0];
  __int128 c = (__int128)m[1][0] * m[2][1] - (__int128)m[1][1] * m[2][0];
  return (__int128)m[0][0] * a - (__int128)m[0][1] * b + (__int128)m[0][2] * c;
}

// One warp per peak; FIT_WARPS warps per CTA; grid (frames, G).
__global__ void __launch_bounds__(FIT_WARPS * 32) k_fit(FitArgs a) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int f = blockIdx.x;
  const int n = min(a.peak_count[f], a.peak_cap);
  const int step = gridDim.y * FIT_WARPS;
  const int n_st = a.rl.n_stx * a.rl.n_sty;
  for (int pi = blockIdx.y * FIT_WARPS + warp; pi < n; pi += step) {
    int4 pk = a.peaks[(size_t)f * a.peak_cap + pi];
    const int ix = pk.x, iy = pk.y, ir = pk.z;
    const uint32_t nv = (uint32_t)pk.w;
    // membership |sqrt(d2) - ir| <= w; integer bounds suffice when w is integral
    const int wi = (int)ceilf(a.w);
    const long long rin = (long long)max(0, ir - wi - 1), rout = (long long)(ir + wi + 1);
    const long long lo2 = (long long)max(0, ir - wi) * max(0, ir - wi), hi2 = (long long)(ir + wi) * (ir + wi);
    long long S[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};  // uu, uv, vv, u, v, n, uz, vz, z
    int sty0 = max(0, (iy - (int)rout) / ST_TH), sty1 = min(a.rl.n_sty - 1, (iy + (int)rout) / ST_TH);
    int stx0 = max(0, (ix - (int)rout) / ST_TW), stx1 = min(a.rl.n_stx - 1, (ix + (int)rout) / ST_TW);
    for (int sty = sty0; sty <= sty1; ++sty)
      for (int stx = stx0; stx <= stx1; ++stx) {
        // skip tiles that cannot meet the annulus
        int bx0 = stx * ST_TW, bx1 = bx0 + ST_TW - 1, by0 = sty * ST_TH, by1 = by0 + ST_TH - 1;
        long long dxn = max(0, max(bx0 - ix, ix - bx1)), dyn = max(0, max(by0 - iy, iy - by1));
        long long dxf = max(abs(ix - bx0), abs(ix - bx1)), dyf = max(abs(iy - by0), abs(iy - by1));
        if (dxn * dxn + dyn * dyn > rout * rout) continue;
        if (dxf * dxf + dyf * dyf < rin * rin) continue;
        size_t tb = (size_t)f * n_st + (size_t)sty * a.rl.n_stx + stx;
        int o0 = a.rl.tile_off[tb], oc = a.rl.tile_cnt[tb];
        for (int j = lane; j < oc; j += 32) {
          uint32_t xy = a.rl.xy[(size_t)f * a.rl.cap + o0 + j];
          int u = (int)(xy & 0xffffu) - ix, v = (int)(xy >> 16) - iy;
          long long d2 = (long long)u * u + (long long)v * v;
          bool in;
          if (a.w_int) {
            in = d2 >= lo2 && d2 <= hi2;
          } else {
            if (d2 < rin * rin || d2 > rout * rout) continue;
            double dist = d_sqrt((double)d2);
            in = fabs(d_sub(dist, (double)ir)) <= (double)a.w;
          }
          if (!in) continue;
          long long z = d2;
          S[0] += (long long)u * u;
          S[1] += (long long)u * v;
          S[2] += (long long)v * v;
          S[3] += u;
          S[4] += v;
          S[5] += 1;
          S[6] += (long long)u * z;
          S[7] += (long long)v * z;
          S[8] += z;
        }
      }
#pragma unroll
    for (int k = 0; k < 9; ++k)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) S[k] += __shfl_xor_sync(0xffffffffu, S[k], o);
    if (lane == 0) {
      rd_ring out;
      out.frame = f;
      out.ix = ix;
      out.iy = iy;
      out.ir = ir;
      out.score = (float)((double)nv / (65536.0 * (double)ir));
      out.n_fit = (int)S[5];
      out.flags = RD_RING_FIT_FAIL;
      out.cx = (float)ix;
      out.cy = (float)iy;
      out.r = (float)ir;
      if (S[5] >= 5) {
        long long M[3][3] = {{S[0], S[1], S[3]}, {S[1], S[2], S[4]}, {S[3], S[4], S[5]}};
        long long rhs[3] = {-S[6], -S[7], -S[8]};
        __int128 det = det3(M);
        if (det != 0) {
          double sol[3];
          for (int c = 0; c < 3; ++c) {
            long long Mc[3][3];
            for (int i = 0; i < 3; ++i)
              for (int j = 0; j < 3; ++j) Mc[i][j] = j == c ? rhs[i] : M[i][j];
            sol[c] = i128_to_double(det3(Mc)) / i128_to_double(det);
          }
          double D = sol[0], E = sol[1], F = sol[2];
          double rr = D * D / 4.0 + E * E / 4.0 - F;
          if (rr > 0.0) {
            out.cx = (float)(ix - D / 2.0);
            out.cy = (float)(iy - E / 2.0);
            out.r = (float)sqrt(rr);
            out.flags = 0;
          }
        }
      }
      int slot = a.offsets[f] + pi;
      if (slot < a.ring_cap)
        a.rings[slot] = out;
      else
        atomicOr(&a.stats->overflow, 8);
    }
  }
}

cudaError_t launch_fit(const FitArgs& a, int4* peaks_mut, int* counts, int* offsets, cudaStream_t st) {
  size_t sm = (size_t)a.peak_cap * 12;
  cudaFuncSetAttribute(k_sort_peaks, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_sort_peaks<<<a.n_frames, SORT_THREADS, sm, st>>>(peaks_mut, a.peak_count, a.peak_cap);
  k_ring_offsets<<<1, 1024, 0, st>>>(a.peak_count, a.n_frames, counts, offsets);
  dim3 grid(a.n_frames, 16);
  k_fit<<<grid, FIT_WARPS * 32, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rd
