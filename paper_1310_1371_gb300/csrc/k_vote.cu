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
#include <algorithm>
#include <climits>

namespace rd {


__device__ __forceinline__ int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Visit the bins that one (ridge pixel, slab, sign) segment can reach: the
// vote positions p + s r X for r in [lo-1, hi+1] lie on a segment; a bin's
// tile collects votes within `halo` px of the tile, and a vote bin is within
// 1/2 px of its real position (1 px margin).
struct SegTiles {
  int tx0, ty0, w, n;  // tiles [tx0, tx0 + w) x [ty0, ty0 + n / w); n = 0 when none
};

// floor(v / T) for v > -4 T (a halo is shorter than a tile): a division by a
// compile-time constant
template <int T>
__device__ __forceinline__ int tile_of(int v) {
  return (int)((unsigned)(v + 4 * T) / (unsigned)T) - 4;
}

template <int T>
__device__ __forceinline__ SegTiles seg_tiles(const BinArgs& a, float px, float py, float dx, float dy, float r0,
                                              float r1, int h) {
  SegTiles t{0, 0, 1, 0};
  // in cells of 2^lc px (a.inv_c = 2^-lc, exact)
  float ax0 = (px + r0 * dx) * a.inv_c, ax1 = (px + r1 * dx) * a.inv_c;
  float ay0 = (py + r0 * dy) * a.inv_c, ay1 = (py + r1 * dy) * a.inv_c;
  int bx0 = (int)floorf(fminf(ax0, ax1)) - 1, bx1 = (int)ceilf(fmaxf(ax0, ax1)) + 1;
  int by0 = (int)floorf(fminf(ay0, ay1)) - 1, by1 = (int)ceilf(fmaxf(ay0, ay1)) + 1;
  bx0 = max(bx0, 0);
  by0 = max(by0, 0);
  bx1 = min(bx1, a.W - 1);
  by1 = min(by1, a.H - 1);
  if (bx0 > bx1 || by0 > by1) return t;
  int tx0 = max(tile_of<T>(bx0 - h), 0), tx1 = min(tile_of<T>(bx1 + h), a.n_atx - 1);
  int ty0 = max(tile_of<T>(by0 - h), 0), ty1 = min(tile_of<T>(by1 + h), a.n_aty - 1);
  t.tx0 = tx0;
  t.ty0 = ty0;
  t.w = tx1 - tx0 + 1;
  t.n = t.w * (ty1 - ty0 + 1);
  return t;
}

// Grid row f handles frame f.  Threads walk the ridge pixels of one slab at a
// time, so the lanes of a warp hold neighbouring pixels, whose segments
// mostly reach the same bins: each step the warp groups equal bins (match)
// and the group leader makes one atomic for the group.  The entry order
// inside a bin is immaterial downstream (votes commute; peaks are sorted
// before the fit).
//
// With a.cta_cnt set (frames of at most BIN_SMEM_MAX bins) the atomics stay
// in shared memory: the count pass counts the CTA's entries per bin of its
// frame and stores them per (bin, CTA); k_bin_cta_scan turns those into each
// CTA's start within the bin and the bin totals; the fill pass starts each
// bin at its offset plus that start, so that every CTA fills a range of its
// own in each bin.
template <bool FILL, int T>
__global__ void __launch_bounds__(256) k_bin(BinArgs a) {
  extern __shared__ int s_bin[];  // per bin of the frame: count (count pass) or next position (fill pass)
  const int lane = threadIdx.x & 31;
  const int gstride = gridDim.x * blockDim.x;
  const int wbase = blockIdx.x * blockDim.x + (threadIdx.x & ~31);
  const int f = blockIdx.y;
  const int cnt = min(a.rl.count[f], a.rl.cap);
  const int nbf = a.n_aty * a.n_atx * a.n_slabs;
  const long long fbin = (long long)f * nbf;
  const bool local = a.cta_cnt != nullptr;
  if (local) {
    if (!FILL) {
      for (int b = threadIdx.x; b < nbf; b += blockDim.x) s_bin[b] = 0;
    } else {
      // the bin's offset plus the frame's earlier CTAs' counts (k_bin_cta_scan)
      for (int b = threadIdx.x; b < nbf; b += blockDim.x)
        s_bin[b] = a.bin_off[fbin + b] + a.cta_cnt[(size_t)(fbin + b) * gridDim.x + blockIdx.x];
    }
    __syncthreads();
  }
  for (int s = 0; s < a.n_slabs; ++s) {
    const int4 sl = a.slabs[s];
    const float r0 = (float)(sl.x - 1), r1 = (float)(sl.y + 1);
    const int h = sl.z;
    for (int base = wbase; base < cnt; base += gstride) {  // warp-uniform
      const int i = base + lane;
      int nb = 0;
      SegTiles t0{0, 0, 1, 0}, t1{0, 0, 1, 0};
      const size_t g = (size_t)f * a.rl.cap + i;
      uint32_t xy = 0;
      float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < cnt) {
        xy = a.rl.xy[g];
        d = a.rl.dir[g];
        const float px = (float)(xy & 0xffffu), py = (float)(xy >> 16);
        t0 = seg_tiles<T>(a, px, py, d.x, d.y, r0, r1, h);
        t1 = seg_tiles<T>(a, px, py, -d.x, -d.y, r0, r1, h);
        nb = t0.n + t1.n;
      }
      const int maxnb = __reduce_max_sync(0xffffffffu, nb);
      for (int k = 0; k < maxnb; ++k) {
        unsigned key = 0xffffffffu;  // bin within the frame
        int sg = 0, tx = 0, ty = 0;
        if (k < nb) {
          sg = k < t0.n ? 0 : 1;
          const SegTiles& t = sg == 0 ? t0 : t1;
          int kk = sg == 0 ? k : k - t0.n;
          ty = t.ty0;
          while (kk >= t.w) {
            kk -= t.w;
            ++ty;
          }
          tx = t.tx0 + kk;
          key = (unsigned)((ty * a.n_atx + tx) * a.n_slabs + s);
          if (!RD_GUARD(tx >= 0 && tx < a.n_atx && ty >= 0 && ty < a.n_aty, a.stats)) key = 0xffffffffu;
        }
        const unsigned grp = __match_any_sync(0xffffffffu, key);
        if (k >= nb || key == 0xffffffffu) continue;
        const int leader = __ffs(grp) - 1;
        const int n_grp = __popc(grp);
        const long long b = fbin + key;
        if (!FILL) {
          if (lane == leader) {
            if (local)
              atomicAdd(&s_bin[key], n_grp);
            else
              atomicAdd(&a.bin_cnt[b], n_grp);
          }
        } else {
          long long first = 0;
          if (lane == leader)
            first = local ? (long long)atomicAdd(&s_bin[key], n_grp)
                          : (long long)a.bin_off[b] + atomicAdd(&a.bin_fill[b], n_grp);
          first = __shfl_sync(grp, first, leader);
          const long long pos = first + __popc(grp & ((1u << lane) - 1u));
          if (pos < a.pool_cap) {
            const float sgn = sg == 0 ? 1.0f : -1.0f;
            // A direction with a component exactly 0 (both parts) is an exact
            // axis: the Hessian's off-diagonal is exactly 0, so the
            // definition's X- is exactly (1, 0) or (0, 1) too (sqrt(x^2) = |x|
            // in binary floating point) and every s r X- is an exact integer.
            const bool axis = (d.x == 0.0f && d.z == 0.0f) || (d.y == 0.0f && d.w == 0.0f);
            const float ex = axis ? (d.x == 0.0f ? 0.0f : 1.0f) : d.x;
            const float ey = axis ? 1.0f - ex : d.y;
            const uint32_t ill = (!axis && a.rl.kvote[g].x > KF_CONST) ? 2u : 0u;
            // position in px relative to the tile region's origin 2^lc (tx T - h, ty T - h)
            const int lx0 = (int)(xy & 0xffffu) - ((tx * T - h) << a.lc);
            const int ly0 = (int)(xy >> 16) - ((ty * T - h) << a.lc);
            a.pool[pos] = make_uint4(((uint32_t)ly0 << 16) | ((uint32_t)lx0 & 0xffffu),
                                     __float_as_uint(sgn * ex), __float_as_uint(sgn * ey),
                                     ((uint32_t)i << 3) | (axis ? 4u : 0u) | ill | (uint32_t)sg);
          }
        }
      }
    }
  }
  if (!FILL && local) {
    __syncthreads();
    for (int b = threadIdx.x; b < nbf; b += blockDim.x)
      a.cta_cnt[(size_t)(fbin + b) * gridDim.x + blockIdx.x] = s_bin[b];
  }
}

// Between the two binning passes with per-CTA counts: one warp per bin turns
// the counts of the frame's gx CTAs (gx <= 64) into exclusive prefixes, in
// place, and writes the bin's total.
__global__ void __launch_bounds__(256) k_bin_cta_scan(int* cta_cnt, int* bin_cnt, long long n_bins, int gx) {
  const long long b = (long long)blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= n_bins) return;
  int* cc = cta_cnt + (size_t)b * gx;
  int carry = 0;
  for (int c0 = 0; c0 < gx; c0 += 32) {
    const int c = c0 + lane;
    const int v = c < gx ? cc[c] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (c < gx) cc[c] = carry + incl - v;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  if (lane == 0) bin_cnt[b] = carry;
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
  L.q = 0;                                                 // int2 (weight, offset) x max_qn (even)
  L.n = round16((size_t)max_qn * 8);                       // u32 x 3 slots x rw2^2
  L.a = L.n + round16(3 * rw2 * rw2 * 4);                  // u32 counts x max_rw^2
  L.hot = L.a + round16((size_t)max_rw * max_rw * 4);      // u16 x 4 x HOT_CAP
  L.total = L.hot + round16((size_t)4 * HOT_CAP * 2);
  return L;
}
size_t vote_smem_bytes(int max_rw, int T, int max_qn) { return vote_smem_layout(max_rw, T, max_qn).total + 64; }

__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc));
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

// A bin entry as a thread holds it across the levels of its slab.
struct VEnt {
  uint32_t xy;     // position relative to the tile region: int16 x | int16 y << 16
  uint32_t ent;    // ridge index << 1 | negative sign
  float X, Y, kf;  // direction (hi parts) and fast-path margin coefficient
};

__device__ __forceinline__ VEnt load_ent(const VoteArgs& a, size_t fbase, long long off, int e) {
  const uint4 E = a.pool[off + e];
  const float sg = (E.w & 1u) ? -1.0f : 1.0f;
  VEnt v;
  v.xy = E.x;
  v.ent = ((E.w >> 3) << 1) | (E.w & 1u);
  v.X = sg * __uint_as_float(E.y);  // back to the unsigned direction
  v.Y = sg * __uint_as_float(E.z);
  // exact axis: every s r X- is an exact integer, decided without a margin
  v.kf = (E.w & 4u) ? -1.0f : ((E.w & 2u) ? 1e30f : KF_CONST);
  return v;
}

constexpr float ROUND_MAGIC = 12582912.0f;  // 1.5 * 2^23: adding it rounds |t| < 2^22 to an integer
constexpr int ROUND_MAGIC_BITS = 0x4B400000;

// Slow path of one vote: double-float refinement, then the double-precision
// definition.  (px, py): the pixel.  Returns (ox, oy, 1 when the FP64
// definition was evaluated).  lc = 0: the vote's bin is p + o.  lc > 0
// (cells of c = 2^lc px): its cell is floor((p + o + c/2) / c).
__device__ __noinline__ int3 vote_bins_slow(const VoteArgs& a, size_t fbase, VEnt v, int px, int py, float rf) {
  const int lc = a.lc;
  const float sr = (v.ent & 1u) ? -rf : rf;
  const size_t g = fbase + (v.ent >> 1);
  const float4 d = a.rl.dir[g];
  const float2 kv = a.rl.kvote[g];
  const int vx = lc ? vote_floor(sr, rf, d.x, d.z, kv.x, kv.y) : vote_offset(sr, rf, d.x, d.z, kv.x, kv.y);
  const int vy = lc ? vote_floor(sr, rf, d.y, d.w, kv.x, kv.y) : vote_offset(sr, rf, d.y, d.w, kv.x, kv.y);
  if (vx != INT_MIN && vy != INT_MIN) return make_int3(vx, vy, 0);
  double X, Y;
  if (a.rl.x64) {  // directed edges: the record keeps the exact double direction
    X = a.rl.x64[g].x;
    Y = a.rl.x64[g].y;
  } else {
    const Eig64 e64 = eigen64(a.rl.hess[3 * g], a.rl.hess[3 * g + 1], a.rl.hess[3 * g + 2], a.D64);
    X = e64.X;
    Y = e64.Y;
  }
  if (X * (double)d.x + Y * (double)d.y < 0.0) {
    X = -X;
    Y = -Y;
  }
  if (lc == 0) return make_int3(vote_bin64(px, (double)sr, X) - px, vote_bin64(py, (double)sr, Y) - py, 1);
  // an offset o with floor((p + o + c/2) / c) = the definition's cell
  const int hc = 1 << (lc - 1);
  return make_int3((vote_cell64(px, (double)sr, X, lc) << lc) - hc - px,
                   (vote_cell64(py, (double)sr, Y, lc) << lc) - hc - py, 1);
}

struct CastCtx {
  int ox0, oy0, RW, h, T;
  int eox, eoy;  // origin the bin entries' positions are relative to
  int lxlo, lxn, lylo, lyn;  // the tile region clipped to the image: [lo, lo + n)
  bool owned;
};

__device__ __forceinline__ int ent_lx(uint32_t xy) { return (int)(int16_t)(xy & 0xffffu); }
__device__ __forceinline__ int ent_ly(uint32_t xy) { return (int)xy >> 16; }

// Bin offsets of one vote by round-to-nearest with the magic constant; the
// result equals the half-up rounding of the double-precision definition when
// the exact remainder is more than the error margin away from 1/2, otherwise
// the slow path decides.  Returns the slab index of the vote or -1.
__device__ __forceinline__ int cast_one(const VoteArgs& a, size_t fbase, const VEnt& v, float rf, const CastCtx& c,
                                        unsigned& nv, unsigned& nfb) {
  const float sr = (v.ent & 1u) ? -rf : rf;
  const float m = __fmaf_rn(rf, v.kf, 1e-10f);
  const float tx = __fmul_rn(sr, v.X), ty = __fmul_rn(sr, v.Y);
  const float fx = __fadd_rn(tx, ROUND_MAGIC), fy = __fadd_rn(ty, ROUND_MAGIC);
  const float dx = __fsub_rn(tx, __fsub_rn(fx, ROUND_MAGIC));  // exact remainder in [-1/2, 1/2]
  const float dy = __fsub_rn(ty, __fsub_rn(fy, ROUND_MAGIC));
  int ox = __float_as_int(fx) - ROUND_MAGIC_BITS;
  int oy = __float_as_int(fy) - ROUND_MAGIC_BITS;
  const int lc = a.lc;
  // lc = 0: round to nearest, certain away from half-integers; lc > 0: floor,
  // certain away from integers
  const bool sure = lc == 0 ? fmaxf(fabsf(dx), fabsf(dy)) < __fsub_rn(0.5f, m) : fminf(fabsf(dx), fabsf(dy)) > m;
  if (!sure) {
    const int3 o = vote_bins_slow(a, fbase, v, ent_lx(v.xy) + (c.eox << lc), ent_ly(v.xy) + (c.eoy << lc), rf);
    nfb += o.z;
    ox = o.x;
    oy = o.y;
  } else if (lc) {
    ox -= dx < 0.0f ? 1 : 0;
    oy -= dy < 0.0f ? 1 : 0;
  }
  const int hc = (1 << lc) >> 1;
  const int lx = ((ent_lx(v.xy) + ox + hc) >> lc) + c.eox - c.ox0;
  const int ly = ((ent_ly(v.xy) + oy + hc) >> lc) + c.eoy - c.oy0;
  if ((unsigned)(lx - c.lxlo) >= (unsigned)c.lxn || (unsigned)(ly - c.lylo) >= (unsigned)c.lyn) return -1;
  if (c.owned && (unsigned)(lx - c.h) < (unsigned)c.T && (unsigned)(ly - c.h) < (unsigned)c.T) ++nv;
  return ly * c.RW + lx;
}

// Dense per-level storage for one bin (used for bins whose hotspots or
// peaks exceed the sparse kernel's capacities).
// The dense kernel works on tiles of T_dense pixels: the bin's own tile, or
// (tiles larger than its storage allows) sub-tile `sub` of a 2 x 2 split.
__device__ __forceinline__ void dense_bin(const VoteArgs& a, int b, int sub, unsigned char* smem) {
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
  const int T = a.T_dense, RW = T + 2 * h, RW2 = T + 2;
  const int H = a.H, W = a.W;
  const int bx0 = tx * a.T + (sub & 1) * T, by0 = ty * a.T + (sub >> 1) * T;  // the (sub-)tile's first pixel
  const unsigned vthr = (unsigned)a.vote_thresh;

  const VoteSmem L = vote_smem_layout(a.max_rw_dense, T, a.max_qn);
  int2* sQq = reinterpret_cast<int2*>(smem + L.q);          // (weight, offset) per window tap
  uint32_t* sN = reinterpret_cast<uint32_t*>(smem + L.n);   // 3 slots of RW2^2 smoothed sums
  uint32_t* sA = reinterpret_cast<uint32_t*>(smem + L.a);   // RW^2 vote counts
  uint16_t* sHot = reinterpret_cast<uint16_t*>(smem + L.hot);  // 4 x HOT_CAP, (vy << 8 | vx)
  const int nA4 = (RW * RW + 3) / 4;
  int* s_nhot = reinterpret_cast<int*>(smem + L.total);          // 4 counters, 4 flags, 2 sums
  int* s_dense = s_nhot + 4;
  unsigned* s_sum = reinterpret_cast<unsigned*>(s_nhot + 8);     // votes, fallbacks of this bin

  if (cnt < cnt_raw && tid == 0) atomicOr(&a.stats->overflow, 2);
  {
    uint4* w4 = reinterpret_cast<uint4*>(sA);
    for (int i = tid; i < nA4; i += VOTE_THREADS) w4[i] = make_uint4(0, 0, 0, 0);
  }
  for (int i = tid; i < 3 * RW2 * RW2; i += VOTE_THREADS) sN[i] = 0;
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) s_nhot[k] = s_dense[k] = 0;
    s_sum[0] = s_sum[1] = 0;
  }
  // per-thread counts, reduced once at the end (a bin's totals fit 32 bits)
  unsigned t_votes = 0, t_fb = 0;

  const size_t fbase = (size_t)f * a.rl.cap;
  const int lv0 = a.r_min - 1;
  // Entry order in a bin follows the ridge list (neighbouring pixels of one
  // arc, whose votes meet), so the lanes of a warp take entries far apart:
  // thread k holds entries k, k + 256, ... in a lane-major numbering.
  const int slot_of_thread = lane * NW + warp;
  VEnt ec[ECACHE];
  int n_cached = 0;
#pragma unroll
  for (int q = 0; q < ECACHE; ++q) {
    int e = q * VOTE_THREADS + slot_of_thread;
    if (e < cnt) {
      ec[q] = load_ent(a, fbase, off, e);
      n_cached = q + 1;
    } else {
      ec[q] = VEnt{0u, 0u, 0.0f, 0.0f, 0.0f};
    }
  }
  const int rounds_extra = max(0, (cnt - ECACHE * VOTE_THREADS + VOTE_THREADS - 1) / VOTE_THREADS);
  CastCtx cc;
  cc.ox0 = bx0 - h;
  cc.oy0 = by0 - h;
  cc.eox = tx * a.T - h;  // the bin's entries are relative to its own region
  cc.eoy = ty * a.T - h;
  cc.RW = RW;
  cc.h = h;
  cc.T = T;
  cc.lxlo = max(0, -cc.ox0);
  cc.lxn = min(RW, W - cc.ox0) - cc.lxlo;
  cc.lylo = max(0, -cc.oy0);
  cc.lyn = min(RW, H - cc.oy0) - cc.lylo;
  __syncthreads();

  for (int r = lo - 1; r <= hi + 1; ++r) {
    const int li = r - lv0;
    const int Rs = a.q_rad[li];
    const int nq = (2 * Rs + 1) * (2 * Rs + 1);
    const int nq2 = (nq + 1) >> 1;  // tap pairs (tables are padded to an even count)
    const int lst = r & 3, slot = r % 3;
    // weights and slab-relative offsets of this level, copied asynchronously
    const int4* gq = reinterpret_cast<const int4*>(a.qq_tab + a.qq_off[s * a.slab_stride + (r - lo + 1)]);
    for (int i = tid; i < nq2; i += VOTE_THREADS) cp_async16(&sQq[2 * i], &gq[i]);
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
    cc.owned = (r >= lo && r <= hi) || (r == lo - 1 && lo == a.r_min) || (r == hi + 1 && hi == a.r_max);
    unsigned nv = 0, nfb = 0;
    const float rf = (float)r;
#pragma unroll
    for (int q = 0; q < ECACHE; ++q) {
      int la = q < n_cached ? cast_one(a, fbase, ec[q], rf, cc, nv, nfb) : -1;
      bool hot = false;
      int vyx = 0;
      if (la >= 0 && RD_GUARD(la < RW * RW, a.stats)) {
        unsigned old = atomicAdd(&sA[la], 1u);
        if (old == vthr) {
          int ly = la / RW, lx = la - ly * RW;
          int vyr = ly - h + 1, vxr = lx - h + 1;
          hot = (unsigned)vyr < (unsigned)RW2 && (unsigned)vxr < (unsigned)RW2;
          vyx = (vyr << 8) | vxr;
        }
      }
      warp_push(hot, (uint16_t)vyx, &s_nhot[lst], sHot + lst * HOT_CAP, HOT_CAP, lane);
    }
    for (int j = 0; j < rounds_extra; ++j) {
      const int e = (ECACHE + j) * VOTE_THREADS + slot_of_thread;
      int la = -1;
      if (e < cnt) {
        VEnt v = load_ent(a, fbase, off, e);
        la = cast_one(a, fbase, v, rf, cc, nv, nfb);
      }
      bool hot = false;
      int vyx = 0;
      if (la >= 0 && RD_GUARD(la < RW * RW, a.stats)) {
        unsigned old = atomicAdd(&sA[la], 1u);
        if (old == vthr) {
          int ly = la / RW, lx = la - ly * RW;
          int vyr = ly - h + 1, vxr = lx - h + 1;
          hot = (unsigned)vyr < (unsigned)RW2 && (unsigned)vxr < (unsigned)RW2;
          vyx = (vyr << 8) | vxr;
        }
      }
      warp_push(hot, (uint16_t)vyx, &s_nhot[lst], sHot + lst * HOT_CAP, HOT_CAP, lane);
    }
    t_votes += nv;
    t_fb += nfb;
    cp_async_wait_all();
    __syncthreads();

    // ---- phase 2: radius-dependent smoothing at this level's hotspots
    uint32_t* cur = sN + slot * RW2 * RW2;
    const int nhot = s_nhot[lst];
    if (cc.owned && tid == 0) {  // algorithmic work counters: each hotspot once
      unsigned long long own = 0;
      for (int v = 0; v < RW2 * RW2; ++v) {
        const int vyr = v / RW2, vxr = v - vyr * RW2;
        const int gx = bx0 - 1 + vxr, gy = by0 - 1 + vyr;
        if (vyr >= 1 && vyr <= T && vxr >= 1 && vxr <= T && gx < W && gy < H &&
            sA[(vyr + h - 1) * RW + (vxr + h - 1)] > vthr)
          ++own;
      }
      if (own) {
        atomicAdd(&a.stats->hotspots, own);
        atomicAdd(&a.stats->smooth_macs, own * (unsigned long long)nq);
      }
    }
    if (tid == 0) {
      // the list of level r - 3 (cleared in phase 1a above) is reused by level r + 1
      s_nhot[(r + 1) & 3] = 0;
      s_dense[(r + 1) & 3] = 0;
    }
    const bool dense = nhot > HOT_CAP;
    if (dense && tid == 0) s_dense[lst] = 1;
    const int ntask = dense ? RW2 * RW2 : nhot;
    const int4* sQ4 = reinterpret_cast<const int4*>(sQq);
    for (int k = warp; k < ntask; k += NW) {
      int vyr, vxr;
      if (!dense) {
        int v = sHot[lst * HOT_CAP + k];
        vyr = v >> 8;
        vxr = v & 0xff;
      } else {
        vyr = k / RW2;
        vxr = k - vyr * RW2;
        int gx = bx0 - 1 + vxr, gy = by0 - 1 + vyr;
        if (gx < 0 || gx >= W || gy < 0 || gy >= H) continue;
        if (sA[(vyr + h - 1) * RW + (vxr + h - 1)] <= vthr) continue;
      }
      const uint32_t* ctr = sA + (vyr + h - 1) * RW + (vxr + h - 1);
      unsigned long long acc0 = 0, acc1 = 0;
      const bool win_ok = RD_GUARD(vyr - 1 + h - Rs >= 0 && vyr - 1 + h + Rs < RW && vxr - 1 + h - Rs >= 0 &&
                                       vxr - 1 + h + Rs < RW,
                                   a.stats);
      for (int q = lane; q < nq2 && win_ok; q += 32) {
        int4 w = sQ4[q];  // two taps: (weight, offset), (weight, offset)
        acc0 += (unsigned long long)(uint32_t)w.x * ctr[w.y];
        acc1 += (unsigned long long)(uint32_t)w.z * ctr[w.w];
      }
      unsigned long long acc = acc0 + acc1;
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
    __syncthreads();

    if (a.dbg_acc && f == 0) {
      for (int v = tid; v < T * T; v += VOTE_THREADS) {
        int iy = v / T, ix = v - iy * T;
        int gx = bx0 + ix, gy = by0 + iy;
        if (gx < W && gy < H) {
          a.dbg_acc[((size_t)li * H + gy) * W + gx] = (int32_t)sA[(iy + h) * RW + (ix + h)];
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
      const bool pdense = s_dense[pl] != 0;
      const int n = pdense ? T * T : s_nhot[pl];
      for (int k = tid; k < n; k += VOTE_THREADS) {
        int iy, ix;
        if (pdense) {
          iy = k / T;
          ix = k - iy * T;
        } else {
          int v = sHot[pl * HOT_CAP + k];
          iy = (v >> 8) - 1;
          ix = (v & 0xff) - 1;
          if (iy < 0 || iy >= T || ix < 0 || ix >= T) continue;
        }
        int gx = bx0 + ix, gy = by0 + iy;
        if (gx >= W || gy >= H) continue;
        int c = (iy + 1) * RW2 + ix + 1;
        unsigned long long nv0 = Nmid[c];
        if (nv0 < thr) continue;
        bool ok = true;
#pragma unroll
        for (int dr = -1; dr <= 1; ++dr) {
          const uint32_t* Lv = dr < 0 ? Nlo : (dr == 0 ? Nmid : Nhi);
          unsigned long long lhs = nv0 * (unsigned long long)(rp + dr);
#pragma unroll
          for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
              if (dr == 0 && dy == 0 && dx == 0) continue;
              unsigned long long rhs = (unsigned long long)Lv[c + dy * RW2 + dx] * (unsigned long long)rp;
              bool precedes = dr < 0 || (dr == 0 && (dy < 0 || (dy == 0 && dx < 0)));
              ok = ok && (precedes ? lhs > rhs : lhs >= rhs);
            }
        }
        if (ok) {
          int kk = atomicAdd(&a.peak_count[f], 1);
          if (kk < a.peak_cap)
            a.peaks[(size_t)f * a.peak_cap + kk] = make_int4(gx << a.lc, gy << a.lc, rp, (int)nv0);
          else
            atomicOr(&a.stats->overflow, 4);
          atomicAdd(&a.stats->peaks, 1ULL);
        }
      }
    }

    // ---- phase 3b: clear the slab for the next level (16-byte stores)
    {
      uint4* w4 = reinterpret_cast<uint4*>(sA);
      for (int i = tid; i < nA4; i += VOTE_THREADS) w4[i] = make_uint4(0, 0, 0, 0);
    }
    __syncthreads();
  }
  {
    const unsigned wv = __reduce_add_sync(0xffffffffu, t_votes), wf = __reduce_add_sync(0xffffffffu, t_fb);
    if (lane == 0 && wv) atomicAdd(&s_sum[0], wv);
    if (lane == 0 && wf) atomicAdd(&s_sum[1], wf);
  }
  __syncthreads();
  if (tid == 0) {
    if (s_sum[0]) atomicAdd(&a.stats->votes, (unsigned long long)s_sum[0]);
    if (s_sum[1]) atomicAdd(&a.stats->fallbacks, (unsigned long long)s_sum[1]);
  }
}

__global__ void __launch_bounds__(VOTE_THREADS, 2) k_vote_dense(VoteArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = min(*a.fb_count, a.fb_cap);
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    __syncthreads();  // the previous bin's readers are done with shared memory
    const int item = a.fb_list[i];
    dense_bin(a, item >> 2, item & 3, smem);
  }
}

// ---- K4 (sparse) --------------------------------------------------------------
// The common path.  Shared memory holds one level of u16 vote counts for the
// tile plus its smoothing halo, the window taps of that level (by rotation
// orbits of four equal weights), and, for the last four levels, the hotspot
// lists with their smoothed sums and a small open-addressing table from
// voxel to list slot: the paper's registering of modified elements, so that
// nothing proportional to the tile area is kept beyond the current level and
// three CTAs fit on an SM with 128-pixel tiles.  A bin whose hotspots, peaks
// or deferred exact votes exceed these capacities emits nothing here and is
// handed to k_vote_dense, which computes the same result with dense
// per-level storage.
constexpr int SP_THREADS = 320;  // 10 warps: three CTAs per SM at 64 registers use 61440 of 65536
constexpr int SP_HOT = 256;     // hotspots per level
constexpr int SP_HASH = 512;    // hash slots per level (power of two, > 2 SP_HOT)
constexpr int SP_PEAKS = 64;    // peaks buffered per CTA
constexpr uint32_t SP_EMPTY = 0xffffffffu;
constexpr int SP_SLOW = 32;     // votes per warp and level left to the exact path after the loop

struct SparseSmem {
  size_t q, a, hash, coord, val, pk, total;
};
__host__ __device__ __forceinline__ SparseSmem sparse_smem_layout(int max_rw, int max_qp) {
  SparseSmem L;
  L.q = 0;                                                        // u32 x max_qp: centre + tap orbits
  L.a = round16((size_t)max_qp * 4);                              // u16 counts x max_rw^2
  L.hash = L.a + round16((((size_t)max_rw * max_rw + 1) / 2) * 4);  // u32 x 4 x SP_HASH
  L.coord = L.hash + (size_t)4 * SP_HASH * 4;                     // u16 x 4 x SP_HOT
  L.val = L.coord + round16((size_t)4 * SP_HOT * 2);              // u32 x 4 x SP_HOT
  L.pk = L.val + (size_t)4 * SP_HOT * 4;                          // int4 x SP_PEAKS
  L.total = L.pk + (size_t)SP_PEAKS * 16;
  return L;
}
size_t sparse_smem_bytes(int max_rw, int max_qp) { return sparse_smem_layout(max_rw, max_qp).total; }

__device__ __forceinline__ uint32_t sp_hash(uint32_t key) { return (key * 2654435761u) >> (32 - 9); }

__device__ __forceinline__ uint32_t sp_lookup(const uint32_t* tab, const uint32_t* val, uint32_t key) {
  uint32_t h = sp_hash(key);
  for (int p = 0; p < SP_HASH; ++p) {
    const uint32_t e = tab[h];
    if (e == SP_EMPTY) return 0u;
    if ((e >> 16) == key) return val[e & 0xffffu];
    h = (h + 1) & (SP_HASH - 1);
  }
  return 0u;
}

// K4 work of one bin b; called by every thread of the CTA.
template <bool COARSE>
__device__ __forceinline__ void vote_bin_sparse(const VoteArgs& a, const int b, unsigned char* smem) {
  const int cnt_raw = a.bin_cnt[b];
  if (cnt_raw == 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int NW = SP_THREADS / 32;
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
  const int ox0 = tx * T - h, oy0 = ty * T - h;
  const int H = a.H, W = a.W;
  // the tile region clipped to the image: [lxlo, lxlo + lxn) x [lylo, lylo + lyn)
  const int lxlo = max(0, -ox0), lxn = min(RW, W - ox0) - lxlo;
  const int lylo = max(0, -oy0), lyn = min(RW, H - oy0) - lylo;
  const unsigned vthr = (unsigned)a.vote_thresh;

  const SparseSmem L = sparse_smem_layout(a.max_rw, a.max_qp);
  uint32_t* sQ = reinterpret_cast<uint32_t*>(smem + L.q);
  uint32_t* sAw = reinterpret_cast<uint32_t*>(smem + L.a);
  const uint16_t* sA16 = reinterpret_cast<const uint16_t*>(sAw);
  uint32_t* sHash = reinterpret_cast<uint32_t*>(smem + L.hash);
  uint16_t* sCoord = reinterpret_cast<uint16_t*>(smem + L.coord);
  uint32_t* sVal = reinterpret_cast<uint32_t*>(smem + L.val);
  int4* sPk = reinterpret_cast<int4*>(smem + L.pk);
  const int nA4 = (((RW * RW + 1) / 2) + 3) / 4;
  __shared__ int s_nhot[4], s_npk, s_abort;
  __shared__ int s_nslow[SP_THREADS / 32], s_slow[SP_THREADS / 32][SP_SLOW];
  __shared__ unsigned s_sum[4];  // votes, fallbacks, owned hotspots, smoothing MACs of this bin
  // per voting level lo-1 .. hi+1 of the slab: R_s, offset of its tap orbits, peak threshold
  __shared__ int s_rad[MAX_SLAB_LEVELS + 2], s_qpo[MAX_SLAB_LEVELS + 2];
  __shared__ unsigned long long s_thr[MAX_SLAB_LEVELS + 2];

  if (cnt < cnt_raw && tid == 0) atomicOr(&a.stats->overflow, 2);
  {
    uint4* w4 = reinterpret_cast<uint4*>(sAw);
    for (int i = tid; i < nA4; i += SP_THREADS) w4[i] = make_uint4(0, 0, 0, 0);
  }
  for (int i = tid; i < 4 * SP_HASH; i += SP_THREADS) sHash[i] = SP_EMPTY;
  if (tid == 0) {
    for (int k = 0; k < 4; ++k) s_nhot[k] = 0;
    s_npk = 0;
    s_abort = a.route_dense;
    for (int k = 0; k < 4; ++k) s_sum[k] = 0;
  }
  if (lane == 0) s_nslow[warp] = 0;
  if (tid <= hi - lo + 2) {
    const int li = lo - 1 + tid - (a.r_min - 1);
    s_rad[tid] = a.q_rad[li];
    s_qpo[tid] = a.qp_off[s * a.slab_stride + tid];
    s_thr[tid] = a.nthr[li];
  }
  // Per-thread counts, reduced once at the end: a bin's totals fit 32 bits
  // (votes and fallbacks <= MAX_SLAB_LEVELS + 2 levels x its entries, MACs <=
  // (MAX_SLAB_LEVELS + 2) x SP_HOT x 81^2).
  unsigned t_votes = 0, t_fb = 0, t_hot = 0, t_macs = 0;
  const size_t fbase = (size_t)f * a.rl.cap;
  const int lv0 = a.r_min - 1;
  const int rounds = (cnt + SP_THREADS - 1) / SP_THREADS;
  const uint4* __restrict__ bin = a.pool + off;  // read-only for the whole kernel
  __syncthreads();

  for (int r = lo - 1; r <= hi + 1 && !s_abort; ++r) {
    const int li = r - lv0;
    const int Rs = s_rad[r - lo + 1];
    const int nq = (2 * Rs + 1) * (2 * Rs + 1);
    const int ng = Rs * (Rs + 1);  // rotation orbits of four taps, after the centre entry
    const int lst = r & 3;
    const uint4* gq = reinterpret_cast<const uint4*>(a.qp_tab + s_qpo[r - lo + 1]);
    for (int i = tid; i <= ng; i += SP_THREADS) cp_async16(&sQ[4 * i], &gq[i]);
    asm volatile("cp.async.commit_group;\n" ::);

    // ---- phase 1: votes of level r; a voxel whose count passes the integer
    //      threshold is registered as a hotspot of this level
    const bool owned = (r >= lo && r <= hi) || (r == lo - 1 && lo == a.r_min) || (r == hi + 1 && hi == a.r_max);
    const float rf = (float)r;
    const float m_r = __fmaf_rn(rf, KF_CONST, 1e-10f);
    const float half_m = __fsub_rn(0.5f, m_r);
    uint32_t* tab = sHash + lst * SP_HASH;
    unsigned nv = 0, nfb = 0;
    uint4 En = make_uint4(0u, 0u, 0u, 0u);  // next round's entry, loaded one round ahead
    if (tid < cnt) En = __ldg(&bin[tid]);
    // One vote into the slab: bounds, ownership count, packed-u16 atomic,
    // hotspot registration on the increment that crosses the threshold.
    auto cast = [&](int lx, int ly) {
      if ((unsigned)(lx - lxlo) >= (unsigned)lxn || (unsigned)(ly - lylo) >= (unsigned)lyn) return;
      nv += (owned && max((unsigned)(lx - h), (unsigned)(ly - h)) < (unsigned)T) ? 1u : 0u;  // inside the tile
      const int la = ly * RW + lx;
      if (!RD_GUARD((unsigned)la < (unsigned)(RW * RW), a.stats)) return;
      const unsigned sh = (la & 1) << 4;
      const unsigned old = (atomicAdd(&sAw[la >> 1], 1u << sh) >> sh) & 0xffffu;
      if (old == vthr) {
        const int vyr = ly - h + 1, vxr = lx - h + 1;
        if ((unsigned)vyr < (unsigned)RW2 && (unsigned)vxr < (unsigned)RW2) {
          const int k = atomicAdd(&s_nhot[lst], 1);
          if (k < SP_HOT) {
            sCoord[lst * SP_HOT + k] = (uint16_t)(((uint32_t)vyr << 8) | (uint32_t)vxr);
          } else {
            s_abort = 1;
          }
        }
      }
    };
    for (int j = 0; j < rounds; ++j) {
      const int e = j * SP_THREADS + tid;
      const uint4 E = En;
      if (e + SP_THREADS < cnt) En = __ldg(&bin[e + SP_THREADS]);
      if (e >= cnt) continue;
      const float tx_ = __fmul_rn(rf, __uint_as_float(E.y)), ty_ = __fmul_rn(rf, __uint_as_float(E.z));
      const float fx = __fadd_rn(tx_, ROUND_MAGIC), fy = __fadd_rn(ty_, ROUND_MAGIC);
      const float dx = __fsub_rn(tx_, __fsub_rn(fx, ROUND_MAGIC));
      const float dy = __fsub_rn(ty_, __fsub_rn(fy, ROUND_MAGIC));
      int ox = __float_as_int(fx) - ROUND_MAGIC_BITS, oy = __float_as_int(fy) - ROUND_MAGIC_BITS;
      // pixels: round to nearest, certain away from half-integers; cells:
      // floor, certain away from integers
      const bool sure = COARSE ? (fminf(fabsf(dx), fabsf(dy)) > m_r || (E.w & 4u)) : fmaxf(fabsf(dx), fabsf(dy)) < half_m;
      if ((E.w & 2u) || !sure) {  // the exact path takes it after the loop
        const int k = atomicAdd(&s_nslow[warp], 1);
        if (k < SP_SLOW)
          s_slow[warp][k] = e;
        else
          s_abort = 1;
        continue;
      }
      if (COARSE) {
        ox -= dx < 0.0f ? 1 : 0;
        oy -= dy < 0.0f ? 1 : 0;
        const int hc = 1 << (a.lc - 1);
        cast((ent_lx(E.x) + ox + hc) >> a.lc, (ent_ly(E.x) + oy + hc) >> a.lc);
      } else {
        cast(ent_lx(E.x) + ox, ent_ly(E.x) + oy);
      }
    }
    __syncwarp();
    {
      const int ns = min(s_nslow[warp], SP_SLOW);
      for (int k = lane; k < ns; k += 32) {
        const uint4 E = __ldg(&bin[s_slow[warp][k]]);
        VEnt v;
        v.xy = E.x;
        v.ent = ((E.w >> 3) << 1) | (E.w & 1u);
        v.X = v.Y = 0.0f;
        v.kf = 0.0f;
        const int3 o = vote_bins_slow(a, fbase, v, ent_lx(E.x) + (ox0 << a.lc), ent_ly(E.x) + (oy0 << a.lc), rf);
        nfb += o.z;
        if (COARSE) {
          const int hc = 1 << (a.lc - 1);
          cast((ent_lx(E.x) + o.x + hc) >> a.lc, (ent_ly(E.x) + o.y + hc) >> a.lc);
        } else {
          cast(ent_lx(E.x) + o.x, ent_ly(E.x) + o.y);
        }
      }
      __syncwarp();
      if (lane == 0) s_nslow[warp] = 0;
    }
    t_votes += nv;
    t_fb += nfb;
    cp_async_wait_all();
    __syncthreads();
    if (s_abort) break;  // uniform: read after the barrier

    // ---- phase 2: hash this level's hotspots (thread per hotspot, starting
    //      with the last warp, which smooths the fewest; the peak tests of
    //      levels r - 1 .. r + 1 look them up after the next barrier) and
    //      smooth at them (warp per hotspot)
    const int nhot = s_nhot[lst];
    {
      unsigned own = 0;
      const int ht = (tid + 32) % SP_THREADS;  // the last warp's lanes take hotspots 0 .. 31
      for (int k = ht; k < nhot; k += SP_THREADS) {
        const uint32_t key = sCoord[lst * SP_HOT + k];
        uint32_t hh = sp_hash(key);
        for (int p = 0; p < SP_HASH; ++p) {
          if (atomicCAS(&tab[hh], SP_EMPTY, (key << 16) | (uint32_t)k) == SP_EMPTY) break;
          hh = (hh + 1) & (SP_HASH - 1);
        }
        const int iy = (int)(key >> 8) - 1, ix = (int)(key & 0xffu) - 1;
        own += ((unsigned)iy < (unsigned)T && (unsigned)ix < (unsigned)T) ? 1u : 0u;
      }
      if (owned) {  // algorithmic work counters: each hotspot once
        t_hot += own;
        t_macs += own * (unsigned)nq;
      }
    }
    // A hotspot takes 8, 16 or 32 lanes, the fewest that hold one orbit
    // each where the window allows (uniform over the level).
    {
      const uint4* sG = reinterpret_cast<const uint4*>(sQ);
      const int lg = ng <= 8 ? 3 : (ng <= 16 ? 4 : 5);
      const int L = 1 << lg, per = 32 >> lg;
      const int sl = lane & (L - 1);
      for (int kb = warp * per; kb < nhot; kb += NW * per) {
        const int k = kb + (lane >> lg);
        unsigned long long acc = 0;
        if (k < nhot) {
          const uint32_t key = sCoord[lst * SP_HOT + k];
          const uint16_t* ctr = sA16 + ((int)(key >> 8) + h - 1) * RW + ((int)(key & 0xffu) + h - 1);
          const int cy = (int)(key >> 8) + h - 1, cxk = (int)(key & 0xffu) + h - 1;
          const bool win_ok = RD_GUARD(cy - Rs >= 0 && cy + Rs < RW && cxk - Rs >= 0 && cxk + Rs < RW, a.stats);
          if (sl == 0 && win_ok) acc = (unsigned long long)sG[0].z * ctr[0];
          for (int q = 1 + sl; q <= ng && win_ok; q += L) {
            const uint4 G = sG[q];
            const int o1 = (int)G.x, o2 = (int)G.y;
            const unsigned c4 = (unsigned)ctr[o1] + (unsigned)ctr[-o1] + (unsigned)ctr[o2] + (unsigned)ctr[-o2];
            acc += (unsigned long long)G.z * c4;
          }
        }
        // Exact sum over the hotspot's lanes in two 32-bit parts: an orbit
        // adds at most 2^16 x 4 x (2^16 - 1) < 2^34 and the centre < 2^32, so
        // a lane's acc < 2^50 for any window that fits in shared memory, and
        // both its low 24 bits and acc >> 24 sum over 32 lanes in 32 bits.
        unsigned s_lo = (unsigned)acc & 0xffffffu, s_hi = (unsigned)(acc >> 24);
        if (lg == 5) {
          s_lo = __reduce_add_sync(0xffffffffu, s_lo);
          s_hi = __reduce_add_sync(0xffffffffu, s_hi);
        } else {
          for (int o = L >> 1; o > 0; o >>= 1) {
            s_lo += __shfl_xor_sync(0xffffffffu, s_lo, o);
            s_hi += __shfl_xor_sync(0xffffffffu, s_hi, o);
          }
        }
        if (sl == 0 && k < nhot) {
          acc = (unsigned long long)s_lo + ((unsigned long long)s_hi << 24);
          if (acc > 0xffffffffULL) {
            atomicOr(&a.stats->overflow, 16);
            acc = 0xffffffffULL;
          }
          sVal[lst * SP_HOT + k] = (uint32_t)acc;
        }
      }
    }
    __syncthreads();

    if (a.dbg_acc && f == 0) {
      for (int v = tid; v < T * T; v += SP_THREADS) {
        const int iy = v / T, ix = v - iy * T;
        const int gx = tx * T + ix, gy = ty * T + iy;
        if (gx < W && gy < H) a.dbg_acc[((size_t)li * H + gy) * W + gx] = (int32_t)sA16[(iy + h) * RW + (ix + h)];
      }
      if (a.dbg_sm) {
        for (int k = tid; k < nhot; k += SP_THREADS) {
          const uint32_t key = sCoord[lst * SP_HOT + k];
          const int iy = (int)(key >> 8) - 1, ix = (int)(key & 0xffu) - 1;
          const int gx = tx * T + ix, gy = ty * T + iy;
          if ((unsigned)iy < (unsigned)T && (unsigned)ix < (unsigned)T && gx < W && gy < H)
            a.dbg_sm[((size_t)li * H + gy) * W + gx] = sVal[lst * SP_HOT + k];
        }
      }
      __syncthreads();  // the capture reads the slab before phase 3 clears it
    }

    // ---- phase 3: peak test of level r - 1 against levels r - 2 .. r; clear
    //      the slab and the registers of level r - 3 for the next level
    const int rp = r - 1;
    if (rp >= lo && rp <= hi) {
      const int pl = rp & 3;
      const int n = s_nhot[pl];
      const unsigned long long thr = s_thr[rp - lo + 1];
      for (int k = tid; k < n; k += SP_THREADS) {
        const uint32_t key = sCoord[pl * SP_HOT + k];
        const int vyr = (int)(key >> 8), vxr = (int)(key & 0xffu);
        const int iy = vyr - 1, ix = vxr - 1;
        if ((unsigned)iy >= (unsigned)T || (unsigned)ix >= (unsigned)T) continue;
        const int gx = tx * T + ix, gy = ty * T + iy;
        if (gx >= W || gy >= H) continue;
        const unsigned long long nv0 = sVal[pl * SP_HOT + k];
        if (nv0 < thr) continue;
        bool ok = true;
        for (int dr = -1; dr <= 1 && ok; ++dr) {
          const int ll = (rp + dr) & 3;
          const unsigned long long lhs = nv0 * (unsigned long long)(rp + dr);
          for (int dy = -1; dy <= 1 && ok; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
              if (dr == 0 && dy == 0 && dx == 0) continue;
              const uint32_t nk = ((uint32_t)(vyr + dy) << 8) | (uint32_t)(vxr + dx);
              const unsigned long long rhs =
                  (unsigned long long)sp_lookup(sHash + ll * SP_HASH, sVal + ll * SP_HOT, nk) * (unsigned long long)rp;
              const bool precedes = dr < 0 || (dr == 0 && (dy < 0 || (dy == 0 && dx < 0)));
              if (precedes ? !(lhs > rhs) : !(lhs >= rhs)) {
                ok = false;
                break;
              }
            }
        }
        if (ok) {
          const int kk = atomicAdd(&s_npk, 1);
          if (kk < SP_PEAKS)
            sPk[kk] = make_int4(gx << a.lc, gy << a.lc, rp, (int)nv0);
          else
            s_abort = 1;
        }
      }
    }
    {
      uint4* w4 = reinterpret_cast<uint4*>(sAw);
      for (int i = tid; i < nA4; i += SP_THREADS) w4[i] = make_uint4(0, 0, 0, 0);
      uint32_t* nt = sHash + ((r + 1) & 3) * SP_HASH;  // level r - 3's table, reused by level r + 1
      for (int i = tid; i < SP_HASH; i += SP_THREADS) nt[i] = SP_EMPTY;
    }
    if (tid == 0) s_nhot[(r + 1) & 3] = 0;
    __syncthreads();
  }
  __syncthreads();
  if (s_abort) {
    if (tid == 0) {
      const int ns = a.T_dense < a.T ? 4 : 1;
      const int k = atomicAdd(a.fb_count, ns);
      for (int j = 0; j < ns; ++j)
        if (k + j < a.fb_cap) a.fb_list[k + j] = b * 4 + j;
    }
    return;
  }
  {
    const unsigned c0 = __reduce_add_sync(0xffffffffu, t_votes), c1 = __reduce_add_sync(0xffffffffu, t_fb);
    const unsigned c2 = __reduce_add_sync(0xffffffffu, t_hot), c3 = __reduce_add_sync(0xffffffffu, t_macs);
    if (lane == 0) {
      if (c0) atomicAdd(&s_sum[0], c0);
      if (c1) atomicAdd(&s_sum[1], c1);
      if (c2) atomicAdd(&s_sum[2], c2);
      if (c3) atomicAdd(&s_sum[3], c3);
    }
  }
  __syncthreads();
  const int npk = s_npk;
  for (int k = tid; k < npk; k += SP_THREADS) {
    const int kk = atomicAdd(&a.peak_count[f], 1);
    if (kk < a.peak_cap)
      a.peaks[(size_t)f * a.peak_cap + kk] = sPk[k];
    else
      atomicOr(&a.stats->overflow, 4);
  }
  if (tid == 0) {
    if (npk) atomicAdd(&a.stats->peaks, (unsigned long long)npk);
    if (s_sum[0]) atomicAdd(&a.stats->votes, (unsigned long long)s_sum[0]);
    if (s_sum[1]) atomicAdd(&a.stats->fallbacks, (unsigned long long)s_sum[1]);
    if (s_sum[2]) atomicAdd(&a.stats->hotspots, (unsigned long long)s_sum[2]);
    if (s_sum[3]) atomicAdd(&a.stats->smooth_macs, (unsigned long long)s_sum[3]);
  }
}

cudaError_t launch_bins(const BinArgs& a, int n_sm, cudaStream_t st, long long n_bins, int* block_sums,
                        long long* total_dev) {
  cudaError_t e;
  // about 8 CTAs per SM in total, split over the frames (grid rows); with
  // per-CTA counts (a.cta_cnt) at most BIN_GRID_MAX CTAs per frame
  int gx = std::max(1, (n_sm * 8 + a.n_frames - 1) / a.n_frames);
  const int nbf = a.n_aty * a.n_atx * a.n_slabs;
  if (a.cta_cnt) gx = std::min(gx, BIN_GRID_MAX);
  const size_t smem = a.cta_cnt ? sizeof(int) * (size_t)nbf : 0;
  const dim3 grid((unsigned)gx, (unsigned)a.n_frames);
  if (a.T == ACC_T)
    k_bin<false, ACC_T><<<grid, 256, smem, st>>>(a);
  else if (a.T == ACC_T_MID)
    k_bin<false, ACC_T_MID><<<grid, 256, smem, st>>>(a);
  else if (a.T == ACC_T_LARGE)
    k_bin<false, ACC_T_LARGE><<<grid, 256, smem, st>>>(a);
  else
    k_bin<false, ACC_T_SMALL><<<grid, 256, smem, st>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.cta_cnt) {
    k_bin_cta_scan<<<(unsigned)((n_bins + 7) / 8), 256, 0, st>>>(a.cta_cnt, a.bin_cnt, n_bins, gx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  int nb = (int)((n_bins + 1023) / 1024);
  k_scan_blocks<<<nb, 1024, 0, st>>>(a.bin_cnt, const_cast<int*>(a.bin_off), block_sums, n_bins);
  k_scan_sums<<<1, 1024, 0, st>>>(block_sums, nb, total_dev);
  k_scan_add<<<nb, 1024, 0, st>>>(const_cast<int*>(a.bin_off), block_sums, n_bins);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (a.T == ACC_T)
    k_bin<true, ACC_T><<<grid, 256, smem, st>>>(a);
  else if (a.T == ACC_T_MID)
    k_bin<true, ACC_T_MID><<<grid, 256, smem, st>>>(a);
  else if (a.T == ACC_T_LARGE)
    k_bin<true, ACC_T_LARGE><<<grid, 256, smem, st>>>(a);
  else
    k_bin<true, ACC_T_SMALL><<<grid, 256, smem, st>>>(a);
  return cudaGetLastError();
}

// K4's work queue: the non-empty bins, largest first (bucketed by the
// leading-zero count of their entry count, i.e. by floor(log2)), so that a
// persistent grid ends with small items.  One CTA; also resets the head.
__global__ void __launch_bounds__(1024) k_queue(const int* bin_cnt, long long n_bins, int* queue, int* n_queue,
                                               int* head) {
  __shared__ int hist[33], start[33];
  const int tid = threadIdx.x;
  if (tid < 33) hist[tid] = 0;
  __syncthreads();
  for (long long b = tid; b < n_bins; b += blockDim.x) {
    const int c = bin_cnt[b];
    if (c > 0) atomicAdd(&hist[__clz(c)], 1);
  }
  __syncthreads();
  if (tid == 0) {
    int sum = 0;
    for (int q = 0; q < 33; ++q) {
      start[q] = sum;
      sum += hist[q];
    }
    *n_queue = sum;
    *head = 0;
  }
  __syncthreads();
  for (long long b = tid; b < n_bins; b += blockDim.x) {
    const int c = bin_cnt[b];
    if (c > 0) queue[atomicAdd(&start[__clz(c)], 1)] = (int)b;
  }
}

// Persistent K4: a fixed grid of CTAs takes bins from the work queue.
// COARSE: cells of 2^a.lc px (a.lc > 0).
template <bool COARSE>
__global__ void __launch_bounds__(SP_THREADS, 3) k_vote(VoteArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  const int n_items = *a.n_queue;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(a.queue_head, 1);
    __syncthreads();  // also: every thread is done with the previous bin's shared memory
    const int item = s_item;
    __syncthreads();  // s_item read by all before thread 0 takes the next item
    if (item >= n_items) break;
    vote_bin_sparse<COARSE>(a, a.queue[item], smem);
  }
}

cudaError_t launch_vote(const VoteArgs& a, long long n_bins, cudaStream_t st) {
  size_t sm = sparse_smem_bytes(a.max_rw, a.max_qp);
  void (*kern)(VoteArgs) = a.lc ? k_vote<true> : k_vote<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_queue<<<1, 1024, 0, st>>>(a.bin_cnt, n_bins, a.queue, a.n_queue, a.queue_head);
  // persistent grid: as many CTAs as are resident at once
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, SP_THREADS, sm) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const unsigned grid = (unsigned)std::max(1LL, std::min<long long>(n_bins, (long long)a.vote_grid * per_sm));
  kern<<<grid, SP_THREADS, sm, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  size_t smd = vote_smem_bytes(a.max_rw_dense, a.T_dense, a.max_qn);
  cudaFuncSetAttribute(k_vote_dense, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smd);
  k_vote_dense<<<(unsigned)a.fb_grid, VOTE_THREADS, smd, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rd
