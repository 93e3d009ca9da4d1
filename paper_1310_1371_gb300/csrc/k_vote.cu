// k_vote.cu -- K3: binning of ridge pixels into (frame, accumulator tile,
// r-slab) bins; K4: ridge-directed voting into a shared-memory accumulator
// and the fused epilogue (hotspot threshold, radius-dependent smoothing, 1/r
// normalisation, float threshold and 3x3x3 local maxima).
//
// Method: Results ("each directed ridge pixel votes ... (x, y) +/- r X-";
// "Local maxima detection in a noisy parameter space": smoothing of each
// equi-radius level with a width proportional to r, 1/r normalisation,
// nearest-neighbour comparison); Methods (sigma(r) = 0.05 r + 0.25); Detailed
// algorithm step 4 (integer hotspot threshold, float threshold as a fraction
// of 2 pi, 3x3x3 box); Additional notes (votes over [r_min - 1, r_max + 1],
// peaks only inside [r_min, r_max]).
//
// The paper streams equi-radius levels through a three-level cyclic buffer.
// Here each CTA owns one x-y tile and one slab of levels: it casts the votes
// of one level into a shared-memory slab (tile plus the smoothing halo), maps
// that level's hotspots into a three-level cyclic buffer of smoothed sums,
// and peak-tests the middle level, so the 3-d accumulator never leaves the SM.
#include "rd_internal.cuh"
#include <climits>

namespace rd {


__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Visit the bins that one (ridge pixel, slab, sign) segment can reach: the
// vote positions p + s r X for r in [lo-1, hi+1] lie on a segment; a bin's
// tile collects votes within `halo` px of the tile, and a vote bin is within
// 1/2 px of its real position (1 px margin).
template <bool FILL>
__global__ void __launch_bounds__(256) k_bin(BinArgs a) {
  const int gstride = gridDim.x * blockDim.x;
  for (int f = 0; f < a.n_frames; ++f) {
    const int cnt = min(a.rl.count[f], a.rl.cap);
    const long long total = (long long)cnt * a.n_slabs;
    for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < total; it += gstride) {
      int i = (int)(it / a.n_slabs), s = (int)(it - (long long)i * a.n_slabs);
      size_t g = (size_t)f * a.rl.cap + i;
      uint32_t xy = a.rl.xy[g];
      float4 d = a.rl.dir[g];
      float px = (float)(xy & 0xffffu), py = (float)(xy >> 16);
      int4 sl = a.slabs[s];
      float r0 = (float)(sl.x - 1), r1 = (float)(sl.y + 1);
      int h = sl.z;
      for (int sg = 0; sg < 2; ++sg) {
        float sgn = sg == 0 ? 1.0f : -1.0f;
        float ax0 = px + sgn * r0 * d.x, ax1 = px + sgn * r1 * d.x;
        float ay0 = py + sgn * r0 * d.y, ay1 = py + sgn * r1 * d.y;
        int bx0 = (int)floorf(fminf(ax0, ax1)) - 1, bx1 = (int)ceilf(fmaxf(ax0, ax1)) + 1;
        int by0 = (int)floorf(fminf(ay0, ay1)) - 1, by1 = (int)ceilf(fmaxf(ay0, ay1)) + 1;
        bx0 = max(bx0, 0);
        by0 = max(by0, 0);
        bx1 = min(bx1, a.W - 1);
        by1 = min(by1, a.H - 1);
        if (bx0 > bx1 || by0 > by1) continue;
        int tx0 = max(floordiv(bx0 - h, a.T), 0), tx1 = min(floordiv(bx1 + h, a.T), a.n_atx - 1);
        int ty0 = max(floordiv(by0 - h, a.T), 0), ty1 = min(floordiv(by1 + h, a.T), a.n_aty - 1);
        for (int ty = ty0; ty <= ty1; ++ty)
          for (int tx = tx0; tx <= tx1; ++tx) {
            long long b = (((long long)f * a.n_aty + ty) * a.n_atx + tx) * a.n_slabs + s;
            if (!FILL) {
              atomicAdd(&a.bin_cnt[b], 1);
            } else {
              long long pos = (long long)a.bin_off[b] + atomicAdd(&a.bin_fill[b], 1);
              if (pos < a.pool_cap) a.pool[pos] = ((uint32_t)i << 1) | (uint32_t)sg;
            }
          }
      }
    }
  }
}

// ---- exclusive scan of int counts (three phases, 1024 per block) ----------
__global__ void k_scan_blocks(const int* in, int* out, int* block_sums, long long n) {
  __shared__ int s[1024];
  long long i = blockIdx.x * 1024LL + threadIdx.x;
  int v = i < n ? in[i] : 0;
  s[threadIdx.x] = v;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
    __syncthreads();
    s[threadIdx.x] += t;
    __syncthreads();
  }
  if (i < n) out[i] = s[threadIdx.x] - v;
  if (threadIdx.x == 1023) block_sums[blockIdx.x] = s[1023];
}

__global__ void k_scan_sums(int* block_sums, int nb, long long* total_out) {
  __shared__ long long s[1024];
  __shared__ long long carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    int i = base + threadIdx.x;
    long long v = i < nb ? block_sums[i] : 0;
    s[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      long long t = threadIdx.x >= o ? s[threadIdx.x - o] : 0;
      __syncthreads();
      s[threadIdx.x] += t;
      __syncthreads();
    }
    long long ex = s[threadIdx.x] - v + carry;
    if (i < nb) block_sums[i] = (int)min(ex, (long long)INT_MAX);
    __syncthreads();
    if (threadIdx.x == 1023) carry += s[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_add(int* out, const int* block_sums, long long n) {
  long long i = blockIdx.x * 1024LL + threadIdx.x;
  if (i < n) out[i] = (int)min((long long)out[i] + block_sums[blockIdx.x], (long long)INT_MAX);
}

// ---- K4 ---------------------------------------------------------------------
// Capacity of the per-level hotspot lists (the paper's registering of
// modified elements).  A level that overflows its list is handled densely
// (same result, slower).
constexpr int HOT_CAP = 768;
constexpr int ECACHE = 4;   // bin entries a thread keeps in registers across levels

// Shared-memory layout of K4; every region starts on a 16-byte boundary.
struct VoteSmem {
  size_t q, n, a, hot, total;
};
__host__ __device__ __forceinline__ size_t round16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ __forceinline__ VoteSmem vote_smem_layout(int max_rw, int T, int max_qn) {
  const size_t rw2 = (size_t)T + 2;
  VoteSmem L;
  L.q = 0;                                                        // int2 (weight, offset) x max_qn
  L.n = round16((size_t)max_qn * 8);                              // u32 x 3 slots x rw2^2
  L.a = L.n + round16(3 * rw2 * rw2 * 4);                         // u16 counts x max_rw^2
  L.hot = L.a + round16((((size_t)max_rw * max_rw + 1) / 2) * 4);  // u16 x 4 x HOT_CAP
  L.total = L.hot + round16((size_t)4 * HOT_CAP * 2);
  return L;
}
size_t vote_smem_bytes(int max_rw, int T, int max_qn) { return vote_smem_layout(max_rw, T, max_qn).total; }

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc));
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::); }

// warp-aggregated append of `val` to list[cap] with counter *cnt
__device__ __forceinline__ void warp_push(bool pred, uint16_t val, int* cnt, uint16_t* list, int cap, int lane) {
  unsigned m = __ballot_sync(0xffffffffu, pred);
  if (!m) return;
  int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(cnt, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) {
    int k = base + __popc(m & ((1u << lane) - 1u));
    if (k < cap) list[k] = val;
  }
}

__device__ __forceinline__ uint32_t a16(const uint32_t* w, int i) { return (w[i >> 1] >> ((i & 1) << 4)) & 0xffffu; }

// A bin entry as a thread holds it across the levels of its slab.
struct VEnt {
  uint32_t xy;     // x | y << 16
  uint32_t ent;    // ridge index << 1 | negative sign
  float X, Y, kf;  // direction (hi parts) and fast-path margin coefficient
};

__device__ __forceinline__ VEnt load_ent(const VoteArgs& a, size_t fbase, long long off, int e) {
  VEnt v;
  v.ent = a.pool[off + e];
  size_t g = fbase + (v.ent >> 1);
  v.xy = a.rl.xy[g];
  float4 d = a.rl.dir[g];
  v.X = d.x;
  v.Y = d.y;
  v.kf = a.rl.kvote[g].x;
  return v;
}

constexpr float ROUND_MAGIC = 12582912.0f;  // 1.5 * 2^23: adding it rounds |t| < 2^22 to an integer
constexpr int ROUND_MAGIC_BITS = 0x4B400000;

// Bin offsets (floor(sr X + 1/2), floor(sr Y + 1/2)) of one vote.  Fast path:
// round to nearest with the magic constant; the result equals the half-up
// rounding of the double-precision definition when the exact remainder is
// more than the error margin away from 1/2.  Otherwise the double-float and
// then the double-precision paths decide.  Returns the number of FP64
// fallbacks taken (0 or 1).
__device__ __forceinline__ int vote_bins(const VoteArgs& a, size_t fbase, const VEnt& v, float rf, int& ox, int& oy) {
  const float sr = (v.ent & 1u) ? -rf : rf;
  const float m = __fmaf_rn(rf, v.kf, 1e-10f);
  const float tx = __fmul_rn(sr, v.X), ty = __fmul_rn(sr, v.Y);
  const float fx = __fadd_rn(tx, ROUND_MAGIC), fy = __fadd_rn(ty, ROUND_MAGIC);
  const float dx = __fsub_rn(tx, __fsub_rn(fx, ROUND_MAGIC));  // exact remainder in [-1/2, 1/2]
  const float dy = __fsub_rn(ty, __fsub_rn(fy, ROUND_MAGIC));
  ox = __float_as_int(fx) - ROUND_MAGIC_BITS;
  oy = __float_as_int(fy) - ROUND_MAGIC_BITS;
  if (__fadd_rn(fabsf(dx), m) < 0.5f && __fadd_rn(fabsf(dy), m) < 0.5f) return 0;
  // slow path: double-float refinement, then the double-precision definition
  const size_t g = fbase + (v.ent >> 1);
  const float4 d = a.rl.dir[g];
  const float2 kv = a.rl.kvote[g];
  int vx = vote_offset(sr, rf, d.x, d.z, kv.x, kv.y);
  int vy = vote_offset(sr, rf, d.y, d.w, kv.x, kv.y);
  if (vx != INT_MIN && vy != INT_MIN) {
    ox = vx;
    oy = vy;
    return 0;
  }
  const int px = (int)(v.xy & 0xffffu), py = (int)(v.xy >> 16);
  Eig64 e64 = eigen64(a.rl.hess[3 * g], a.rl.hess[3 * g + 1], a.rl.hess[3 * g + 2], a.D64);
  double X = e64.X, Y = e64.Y;
  if (X * (double)d.x + Y * (double)d.y < 0.0) {
    X = -X;
    Y = -Y;
  }
  ox = vote_bin64(px, (double)sr, X) - px;
  oy = vote_bin64(py, (double)sr, Y) - py;
  return 1;
}

__global__ void __launch_bounds__(VOTE_THREADS, 2) k_vote(VoteArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x;
  const int cnt_raw = a.bin_cnt[b];
  if (cnt_raw == 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NW = VOTE_THREADS / 32;
  int t = b;
  const int s = t % a.n_slabs;
  t /= a.n_slabs;
  const int tx = t % a.n_atx;
  t /= a.n_atx;
  const int ty = t % a.n_aty;
  const int f = t / a.n_aty;
  const long long off = a.bin_off[b];
  const int cnt = (int)max(0LL, min((long long)cnt_raw, a.pool_cap - off));
  const int4 sl = a.slabs[s];
  const int lo = sl.x, hi = sl.y, h = sl.z;
  const int T = a.T, RW = T + 2 * h, RW2 = T + 2;
  const int ox0 = tx * T - h, oy0 = ty * T - h;  // image coords of the slab's (0, 0)
  const int H = a.H, W = a.W;
  const unsigned vthr = (unsigned)a.vote_thresh;

  const VoteSmem L = vote_smem_layout(a.max_rw, T, a.max_qn);
  int2* sQq = reinterpret_cast<int2*>(smem + L.q);                             // max_qn (weight, offset)
  uint32_t* sN = reinterpret_cast<uint32_t*>(smem + L.n);                      // 3 slots of RW2^2
  uint32_t* sAw = reinterpret_cast<uint32_t*>(smem + L.a);                     // RW^2 u16 counts
  const int nAw4 = (((RW * RW + 1) / 2) + 3) / 4;                              // uint4 words in use (<= region)
  uint16_t* sHot = reinterpret_cast<uint16_t*>(smem + L.hot);                  // 4 x HOT_CAP, (vy << 8 | vx)
  __shared__ int s_nhot[4], s_dense[4];
  __shared__ unsigned long long s_votes, s_fb;

  if (cnt < cnt_raw && tid == 0) atomicOr(&a.stats->overflow, 2);
  {
    uint4* w4 = reinterpret_cast<uint4*>(sAw);
    for (int i = tid; i < nAw4; i += VOTE_THREADS) w4[i] = make_uint4(0, 0, 0, 0);
  }
  for (int i = tid; i < 3 * RW2 * RW2; i += VOTE_THREADS) sN[i] = 0;
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) s_nhot[k] = s_dense[k] = 0;
    s_votes = 0;
    s_fb = 0;
  }

  const size_t fbase = (size_t)f * a.rl.cap;
  const int lv0 = a.r_min - 1;
  const int rounds = (cnt + VOTE_THREADS - 1) / VOTE_THREADS;
  VEnt ec[ECACHE];
#pragma unroll
  for (int j = 0; j < ECACHE; ++j) {
    int e = j * VOTE_THREADS + tid;
    if (e < cnt) ec[j] = load_ent(a, fbase, off, e);
    else ec[j] = VEnt{0u, 0u, 0.0f, 0.0f, 0.0f};
  }
  __syncthreads();

  for (int r = lo - 1; r <= hi + 1; ++r) {
    const int li = r - lv0;
    const int Rs = a.q_rad[li];
    const int nq = (2 * Rs + 1) * (2 * Rs + 1);
    const int lst = r & 3, slot = r % 3;
    // weights and slab-relative offsets of this level, copied asynchronously
    const int2* gq = a.qq_tab + a.qq_off[s * (SLAB_LEVELS + 2) + (r - lo + 1)];
    for (int i = tid; i < nq; i += VOTE_THREADS) cp_async8(&sQq[i], &gq[i]);
    asm volatile("cp.async.commit_group;\n" ::);

    // ---- phase 1a: clear level r-3's smoothed sums out of the slot
    {
      const int ol = (r + 1) & 3;  // list of level r - 3
      uint32_t* os = sN + slot * RW2 * RW2;
      if (s_dense[ol]) {
        for (int i = tid; i < RW2 * RW2; i += VOTE_THREADS) os[i] = 0;
      } else {
        const int n = s_nhot[ol];
        for (int k = tid; k < n; k += VOTE_THREADS) {
          int v = sHot[ol * HOT_CAP + k];
          os[(v >> 8) * RW2 + (v & 0xff)] = 0;
        }
      }
    }

    // ---- phase 1b: cast this level's votes into the slab
    const bool owned = (r >= lo && r <= hi) || (r == lo - 1 && lo == a.r_min) || (r == hi + 1 && hi == a.r_max);
    unsigned nv = 0, nfb = 0;
    const float rf = (float)r;
    for (int j = 0; j < rounds; ++j) {
      const int e = j * VOTE_THREADS + tid;
      const bool valid = e < cnt;
      VEnt v;
      if (j < ECACHE) {
#pragma unroll
        for (int q = 0; q < ECACHE; ++q)
          if (q == j) v = ec[q];
      } else {
        v = valid ? load_ent(a, fbase, off, e) : VEnt{0u, 0u, 0.0f, 0.0f, 0.0f};
      }
      bool hit = false;
      int la = 0;
      if (valid) {
        int vx, vy;
        nfb += vote_bins(a, fbase, v, rf, vx, vy);
        const int bx = (int)(v.xy & 0xffffu) + vx, by = (int)(v.xy >> 16) + vy;
        const int lx = bx - ox0, ly = by - oy0;
        if ((unsigned)bx < (unsigned)W && (unsigned)by < (unsigned)H && (unsigned)lx < (unsigned)RW &&
            (unsigned)ly < (unsigned)RW) {
          hit = true;
          la = ly * RW + lx;
          if (owned && (unsigned)(lx - h) < (unsigned)T && (unsigned)(ly - h) < (unsigned)T) ++nv;
        }
      }
      unsigned oldc = 0;
      if (hit) {
        unsigned sh = (la & 1) << 4;
        oldc = (atomicAdd(&sAw[la >> 1], 1u << sh) >> sh) & 0xffffu;
      }
      int vyr = 0, vxr = 0;
      bool hot = false;
      if (hit && oldc == vthr) {
        int ly = la / RW, lx = la - ly * RW;
        vyr = ly - h + 1;
        vxr = lx - h + 1;
        hot = vyr >= 0 && vyr < RW2 && vxr >= 0 && vxr < RW2;
      }
      warp_push(hot, (uint16_t)((vyr << 8) | vxr), &s_nhot[lst], sHot + lst * HOT_CAP, HOT_CAP, lane);
    }
    if (nv) atomicAdd(&s_votes, (unsigned long long)nv);
    if (nfb) atomicAdd(&s_fb, (unsigned long long)nfb);
    cp_async_wait_all();
    __syncthreads();

    // ---- phase 2: radius-dependent smoothing at this level's hotspots
    uint32_t* cur = sN + slot * RW2 * RW2;
    const int nhot = s_nhot[lst];
    if (tid == 0) {
      // the list of level r - 3 (cleared in phase 1a above) is reused by level r + 1
      s_nhot[(r + 1) & 3] = 0;
      s_dense[(r + 1) & 3] = 0;
    }
    if (nhot <= HOT_CAP) {
      for (int k = warp; k < nhot; k += NW) {
        int v = sHot[lst * HOT_CAP + k];
        int vyr = v >> 8, vxr = v & 0xff;
        int center = (vyr + h - 1) * RW + (vxr + h - 1);
        unsigned long long acc = 0;
        for (int q = lane; q < nq; q += 32) {
          int2 w = sQq[q];
          acc += (unsigned long long)(uint32_t)w.x * a16(sAw, center + w.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
          if (acc > 0xffffffffULL) {
            atomicOr(&a.stats->overflow, 16);
            acc = 0xffffffffULL;
          }
          cur[vyr * RW2 + vxr] = (uint32_t)acc;
        }
      }
    } else {
      // dense fallback: every in-image voxel of the ring region
      if (tid == 0) s_dense[lst] = 1;
      for (int v = warp; v < RW2 * RW2; v += NW) {
        int vyr = v / RW2, vxr = v - vyr * RW2;
        int gx = tx * T - 1 + vxr, gy = ty * T - 1 + vyr;
        if (gx < 0 || gx >= W || gy < 0 || gy >= H) continue;
        int center = (vyr + h - 1) * RW + (vxr + h - 1);
        if (a16(sAw, center) <= vthr) continue;
        unsigned long long acc = 0;
        for (int q = lane; q < nq; q += 32) {
          int2 w = sQq[q];
          acc += (unsigned long long)(uint32_t)w.x * a16(sAw, center + w.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
          if (acc > 0xffffffffULL) {
            atomicOr(&a.stats->overflow, 16);
            acc = 0xffffffffULL;
          }
          cur[v] = (uint32_t)acc;
        }
      }
    }
    __syncthreads();

    if (a.dbg_acc && f == 0) {
      for (int v = tid; v < T * T; v += VOTE_THREADS) {
        int iy = v / T, ix = v - iy * T;
        int gx = tx * T + ix, gy = ty * T + iy;
        if (gx < W && gy < H) {
          a.dbg_acc[((size_t)li * H + gy) * W + gx] = (int32_t)a16(sAw, (iy + h) * RW + (ix + h));
          if (a.dbg_sm) a.dbg_sm[((size_t)li * H + gy) * W + gx] = cur[(iy + 1) * RW2 + ix + 1];
        }
      }
      __syncthreads();  // the capture reads the slab before phase 3b clears it
    }

    // ---- phase 3a: peak test of level r - 1 (levels r - 2, r - 1, r are in the slots)
    const int rp = r - 1;
    if (rp >= lo && rp <= hi) {
      const uint32_t* Nlo = sN + ((rp + 2) % 3) * RW2 * RW2;
      const uint32_t* Nmid = sN + (rp % 3) * RW2 * RW2;
      const uint32_t* Nhi = cur;
      const unsigned long long thr = a.nthr[rp - lv0];
      const int pl = rp & 3;
      const bool dense = s_dense[pl] != 0;
      const int n = dense ? T * T : s_nhot[pl];
      for (int k = tid; k < n; k += VOTE_THREADS) {
        int iy, ix;
        if (dense) {
          iy = k / T;
          ix = k - iy * T;
        } else {
          int v = sHot[pl * HOT_CAP + k];
          iy = (v >> 8) - 1;
          ix = (v & 0xff) - 1;
          if (iy < 0 || iy >= T || ix < 0 || ix >= T) continue;
        }
        int gx = tx * T + ix, gy = ty * T + iy;
        if (gx >= W || gy >= H) continue;
        int c = (iy + 1) * RW2 + ix + 1;
        unsigned long long nv0 = Nmid[c];
        if (nv0 < thr) continue;
        bool ok = true;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
          const uint32_t* L = dr < 0 ? Nlo : (dr == 0 ? Nmid : Nhi);
          unsigned long long lhs = nv0 * (unsigned long long)(rp + dr);
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              if (dr == 0 && dy == 0 && dx == 0) continue;
              unsigned long long rhs = (unsigned long long)L[c + dy * RW2 + dx] * (unsigned long long)rp;
              bool precedes = dr < 0 || (dr == 0 && (dy < 0 || (dy == 0 && dx < 0)));
              ok = ok && (precedes ? lhs > rhs : lhs >= rhs);
            }
        }
        if (ok) {
          int kk = atomicAdd(&a.peak_count[f], 1);
          if (kk < a.peak_cap)
            a.peaks[(size_t)f * a.peak_cap + kk] = make_int4(gx, gy, rp, (int)nv0);
          else
            atomicOr(&a.stats->overflow, 4);
          atomicAdd(&a.stats->peaks, 1ULL);
        }
      }
    }

    // ---- phase 3b: clear the slab for the next level (16-byte stores)
    {
      uint4* w4 = reinterpret_cast<uint4*>(sAw);
      for (int i = tid; i < nAw4; i += VOTE_THREADS) w4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (s_votes) atomicAdd(&a.stats->votes, s_votes);
    if (s_fb) atomicAdd(&a.stats->fallbacks, s_fb);
  }
}

cudaError_t launch_bins(const BinArgs& a, int n_sm, cudaStream_t st, long long n_bins, int* block_sums,
                        long long* total_dev) {
  cudaError_t e;
  k_bin<false><<<n_sm * 8, 256, 0, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  int nb = (int)((n_bins + 1023) / 1024);
  k_scan_blocks<<<nb, 1024, 0, st>>>(a.bin_cnt, const_cast<int*>(a.bin_off), block_sums, n_bins);
  k_scan_sums<<<1, 1024, 0, st>>>(block_sums, nb, total_dev);
  k_scan_add<<<nb, 1024, 0, st>>>(const_cast<int*>(a.bin_off), block_sums, n_bins);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_bin<true><<<n_sm * 8, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_vote(const VoteArgs& a, long long n_bins, cudaStream_t st) {
  size_t sm = vote_smem_bytes(a.max_rw, a.T, a.max_qn);
  cudaFuncSetAttribute(k_vote, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_vote<<<(unsigned)n_bins, VOTE_THREADS, sm, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rd
