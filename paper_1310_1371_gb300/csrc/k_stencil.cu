// k_stencil.cu -- K1: fused Gaussian smoothing, second-order Sobel Hessian,
// principal curvature k- and direction X-, and the directed-ridge mask, in
// one pass over the frame (compiled with EDGE: the directed-edge variant of
// the Additional notes, the gradient in place of the Hessian); K2:
// double-float refinement of X- per ridge pixel.
//
// Method: Methods ("Algorithm implementation": Gaussian convolution, then the
// 5x5 second-order Sobel operator); Results ("Directed ridge detection &
// votes collection": k- < 0 and a local minimum along X-); Detailed algorithm,
// steps 1-2 (k- below a curvature threshold tau <= 0, X- computed for those
// pixels, local-minimum test along X-, ridge coordinates recorded).
#include "rd_internal.cuh"
#include "rd_cert.cuh"
#include <climits>
#include <type_traits>

namespace rd {


// reflect-101 index (valid outputs only ever need one reflection; far
// indices, used only by discarded outputs of partial tiles, are clamped)
__device__ __forceinline__ int reflect101(int i, int n) {
  i = i < 0 ? -i : i;
  i = i >= n ? 2 * (n - 1) - i : i;
  return min(max(i, 0), n - 1);
}


// Exact Hessian H' = 64 S^2 (Lxx, Lyy, Lxy) at Hessian-tile coordinates
// (hy, hx): the 5x5 second-order Sobel stencils of the exact smoothed tile
// L' (u64, row stride PW), whose rows hy .. hy + 4 and columns hx .. hx + 4
// it reads.
__device__ __forceinline__ void hess_exact(const unsigned long long* sL, int PW, int hy, int hx, long long& hxx,
                                           long long& hyy, long long& hxy) {
  const long long s5[5] = {1, 4, 6, 4, 1}, d2[5] = {1, 0, -2, 0, 1}, d1[5] = {-1, -2, 0, 2, 1};
  hxx = hyy = hxy = 0;
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const long long* row = reinterpret_cast<const long long*>(sL) + (hy + dy) * PW + hx;
    const long long l0 = row[0], l1 = row[1], l2 = row[2], l3 = row[3], l4 = row[4];
    const long long sx = l0 + 4 * (l1 + l3) + 6 * l2 + l4;
    const long long d2x = l0 - 2 * l2 + l4;
    const long long d1x = (l4 - l0) + 2 * (l3 - l1);
    hxx += s5[dy] * d2x;
    hyy += d2[dy] * sx;
    hxy += d1[dy] * d1x;
  }
}

// Exact first-order 5x5 Sobel of L' at Hessian-tile coordinates (hy, hx):
// (Gx', Gy') = 128 S^2 (Gx, Gy).
__device__ __forceinline__ void grad_exact(const unsigned long long* sL, int PW, int hy, int hx, long long& gx,
                                           long long& gy) {
  const long long s5[5] = {1, 4, 6, 4, 1}, d1[5] = {-1, -2, 0, 2, 1};
  gx = gy = 0;
#pragma unroll
  for (int dy = 0; dy < 5; ++dy) {
    const long long* row = reinterpret_cast<const long long*>(sL) + (hy + dy) * PW + hx;
    const long long l0 = row[0], l1 = row[1], l2 = row[2], l3 = row[3], l4 = row[4];
    const long long sx = l0 + 4 * (l1 + l3) + 6 * l2 + l4;
    const long long d1x = (l4 - l0) + 2 * (l3 - l1);
    gx += s5[dy] * d1x;
    gy += d1[dy] * sx;
  }
}

// The directed-edge definition in double precision (Additional notes: the
// gradient replaces the Hessian): (Gx, Gy) = (Gx', Gy') / D, |grad| =
// sqrt(Gx^2 + Gy^2), and where |grad| > thresh (and > 0) the unit direction
// with X > 0 or (X = 0 and Y > 0), else (0, 0); one correctly rounded
// operation per step.
struct Grad64 {
  double g, X, Y;
};
__device__ __forceinline__ Grad64 grad64(long long gx, long long gy, double D, double thresh) {
  const double Gx = d_div(__ll2double_rn(gx), D), Gy = d_div(__ll2double_rn(gy), D);
  Grad64 r;
  r.g = d_sqrt(d_add(d_mul(Gx, Gx), d_mul(Gy, Gy)));
  r.X = r.Y = 0.0;
  if (r.g != 0.0 && r.g > thresh) {
    r.X = d_div(Gx, r.g);
    r.Y = d_div(Gy, r.g);
    if (r.X < 0.0 || (r.X == 0.0 && r.Y < 0.0)) {
      r.X = -r.X;
      r.Y = -r.Y;
    }
  }
  return r;
}

// Pixels per step of the exact test (9 threads each).
constexpr int FB_CHUNK = ST_THREADS / 9;

// FP32 gradient (Gx, Gy) = fl(G') x fl(1/D) from the row filters of five
// consecutive rows: the column filter s of the d1 rows, and d1 of the s rows.
__device__ __forceinline__ void grad32_v(float x0, float x1, float x2, float x3, float x4, float y0, float y1, float y3,
                                         float y4, float invD, float& gx, float& gy) {
  const float Gx = __fmaf_rn(6.0f, x2, __fmaf_rn(4.0f, __fadd_rn(x1, x3), __fadd_rn(x0, x4)));
  const float Gy = __fmaf_rn(2.0f, __fsub_rn(y3, y1), __fsub_rn(y4, y0));
  gx = __fmul_rn(Gx, invD);
  gy = __fmul_rn(Gy, invD);
}

// Shared-memory layout of K1 (byte offsets, all 8-byte aligned): the exact
// smoothed tile L' (u64, alive to the end), one region holding first the
// input tile and the horizontal pass (u32) and then the FP32 Hessian
// entries (or gradient) of L, the rounded L (f32) whose bytes later hold the
// pixel lists, k- and its error bound (f32), and the compaction scratch.
struct StencilSmem {
  unsigned l, x, f, k, scan, total;
};
// The input tile is stored as u16 from column x0 - ORG, ORG = HALO rounded
// up to 16 pixels, so that interior tiles fill whole rows with aligned
// 16-byte copies; its row stride is a multiple of 8 elements (16 bytes).
// The horizontal pass's row stride is a multiple of 4, so that a thread's
// four outputs go out as one 16-byte store.
constexpr __host__ __device__ int in_org(int halo) { return (halo + 15) & ~15; }
constexpr __host__ __device__ int in_stride(int halo) { return ST_TW + 2 * in_org(halo) + 8; }
constexpr int P_STRIDE = ST_TW + 8;  // >= ST_TW + 6 outputs, a multiple of 4
// Rows per thread of the vertical pass, and the horizontal pass's spare rows
// that its last window reads past the tile (outputs not stored).
constexpr int C_RUN = 7;
constexpr int C_SPARE = (ST_TH + 6 + C_RUN - 1) / C_RUN * C_RUN - (ST_TH + 6);

__host__ __device__ __forceinline__ StencilSmem stencil_smem_layout(int R) {
  const int HALO = R + 3;
  const unsigned IW = in_stride(HALO), IH = ST_TH + 2 * HALO;
  const unsigned PW = ST_TW + 6, LH = ST_TH + 6;
  const unsigned HW2 = ST_TW + 2, HH2 = ST_TH + 2;
  // the horizontal pass has C_SPARE spare rows that the vertical pass's last
  // window may read (their outputs are not stored)
  const unsigned in_bytes = ((IH * IW * 2 + 15) & ~15u) + (IH + C_SPARE) * P_STRIDE * 4,
                 hf_bytes = 3 * HH2 * HW2 * 4;
  const unsigned lf_bytes = LH * PW * 4, list_bytes = ST_TW * ST_TH * (1 + 2 + 2);
  StencilSmem L;
  L.l = 0;
  L.x = LH * PW * 8;
  L.f = L.x + (((in_bytes > hf_bytes ? in_bytes : hf_bytes) + 15) & ~15u);
  L.k = L.f + (((lf_bytes > list_bytes ? lf_bytes : list_bytes) + 15) & ~15u);
  L.scan = L.k + 2 * HH2 * HW2 * 4;
  L.total = L.scan + (ST_THREADS / 32 + 1) * 4;
  return L;
}

// Widen 16 bytes of u8 pixels to 16 u16 (two 16-byte halves).
__device__ __forceinline__ void widen_u8(uint4 q, uint4& lo, uint4& hi) {
  lo = make_uint4(__byte_perm(q.x, 0u, 0x4140), __byte_perm(q.x, 0u, 0x4342), __byte_perm(q.y, 0u, 0x4140),
                  __byte_perm(q.y, 0u, 0x4342));
  hi = make_uint4(__byte_perm(q.z, 0u, 0x4140), __byte_perm(q.z, 0u, 0x4342), __byte_perm(q.w, 0u, 0x4140),
                  __byte_perm(q.w, 0u, 0x4342));
}

// Largest of the eight u16 in a 16-byte vector.
__device__ __forceinline__ uint32_t max_u16x8(uint4 q) {
  const uint32_t m = __vmaxu2(__vmaxu2(q.x, q.y), __vmaxu2(q.z, q.w));
  return max(m & 0xffffu, m >> 16);
}

// RC > 0: the Gaussian half-width R is the compile-time RC (taps unrolled,
// several outputs per thread from register windows); RC = 0: R from the taps.
// EDGE: directed edges (Additional notes) -- the gradient replaces the
// Hessian and -|grad| takes the place of k- in every test below.
template <typename Tin, int RC, bool EDGE>
__global__ void __launch_bounds__(ST_THREADS, 5) k_stencil_ridge(StencilArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int R = RC > 0 ? RC : a.taps.R;
  const int HALO = R + 3;
  const int IW = in_stride(HALO), IH = ST_TH + 2 * HALO, ORG = in_org(HALO);
  const int PW = ST_TW + 6, PWs = P_STRIDE, LH = ST_TH + 6;
  const int HW2 = ST_TW + 2, HH2 = ST_TH + 2;
  const int H = a.H, W = a.W;

  // shared memory carve-up (8-byte aligned pieces first).  The input tile
  // and the horizontal pass (sI, sP) are dead once the vertical pass is
  // done, and the FP32 Hessian entries are written after it, so they share
  // bytes; the rounded L is dead after the Hessian pass and its bytes take
  // the pixel lists.
  const StencilSmem Ls = stencil_smem_layout(R);
  unsigned long long* sL = reinterpret_cast<unsigned long long*>(smem + Ls.l);  // LH*PW
  uint16_t* sI = reinterpret_cast<uint16_t*>(smem + Ls.x);                     // IH*IW, from column x0 - ORG
  uint32_t* sP = reinterpret_cast<uint32_t*>(smem + Ls.x + ((IH * IW * 2 + 15) & ~15));  // IH*PWs
  float* sHa = reinterpret_cast<float*>(smem + Ls.x);                          // HH2*HW2 each
  float* sHb = sHa + HH2 * HW2;
  float* sHc = sHb + HH2 * HW2;
  float* sLf = reinterpret_cast<float*>(smem + Ls.f);                          // LH*PW
  uint16_t* sU = reinterpret_cast<uint16_t*>(smem + Ls.f);                     // undecided pixels
  uint16_t* sR = sU + ST_TW * ST_TH;                                           // ridge pixels
  uint8_t* sV = reinterpret_cast<uint8_t*>(sR + ST_TW * ST_TH);                // exact verdicts
  float* sK = reinterpret_cast<float*>(smem + Ls.k);                           // HH2*HW2
  float* sE = sK + HH2 * HW2;
  int* sScan = reinterpret_cast<int*>(smem + Ls.scan);                         // warps + 1
  __shared__ int32_t q[2 * MAX_RG + 1];
  __shared__ unsigned s_lmax;  // bits of the largest rounded L of the tile (all >= 0)
  __shared__ int s_nu;
  __shared__ unsigned s_imax;  // largest input value of the tile and its halo
  __shared__ int s_ncand;      // pixels listed for the direction test

  if (tid < 2 * R + 1) q[tid] = a.taps.q[tid];
  if (tid == 0) {
    s_lmax = 0u;
    s_nu = 0;
    s_imax = 0u;
    s_ncand = 0;
  }

  const int f = blockIdx.z;
  const int x0 = blockIdx.x * ST_TW, y0 = blockIdx.y * ST_TH;
  const Tin* img = reinterpret_cast<const Tin*>(a.frames) + (size_t)f * H * W;

  // ---- A: input tile with reflect-101 halo.  Interior tiles of frames
  //      whose rows are 16-byte aligned copy the aligned span [x0 - ORG,
  //      x0 + ST_TW + ORG) of each row with 16-byte loads; other tiles load
  //      pixel by pixel, reflecting at the borders, one row per warp step.
  {
    const int lane = tid & 31, warp = tid >> 5;
    const bool interior = x0 >= HALO && y0 >= HALO && x0 + ST_TW + HALO <= W && y0 + ST_TH + HALO <= H;
    const bool vec = a.vec_rows && y0 >= HALO && y0 + ST_TH + HALO <= H && x0 >= ORG && x0 + ST_TW + ORG <= W;
    const int IWn = ST_TW + 2 * HALO;  // columns used
    const int coff = ORG - HALO;       // column of x0 - HALO in the tile
    uint32_t vmax = 0u;
    if (vec) {
      constexpr int VEC = 16 / (int)sizeof(Tin);  // pixels per 16-byte load
      const int NV = (ST_TW + 2 * ORG) / VEC;     // loads per row
      constexpr int NIT = 3;                      // loads per thread in flight (>= 54 rows x 8 / 256)
      for (int base = 0; base < IH * NV; base += NIT * ST_THREADS) {
        uint4 q[NIT];
#pragma unroll
        for (int u = 0; u < NIT; ++u) {
          const int it = min(base + u * ST_THREADS + tid, IH * NV - 1);
          const int iy = it / NV, v = it - iy * NV;
          const Tin* src = img + (size_t)(y0 - HALO + iy) * W + (x0 - ORG) + v * VEC;
          q[u] = __ldg(reinterpret_cast<const uint4*>(src));
        }
#pragma unroll
        for (int u = 0; u < NIT; ++u) {
          const int it = base + u * ST_THREADS + tid;
          if (it >= IH * NV) continue;
          const int iy = it / NV, v = it - iy * NV;
          uint16_t* dst = sI + iy * IW + v * VEC;
          if constexpr (sizeof(Tin) == 1) {
            uint4 lo, hi;
            widen_u8(q[u], lo, hi);
            reinterpret_cast<uint4*>(dst)[0] = lo;
            reinterpret_cast<uint4*>(dst)[1] = hi;
          } else {
            reinterpret_cast<uint4*>(dst)[0] = q[u];
            vmax = max(vmax, max_u16x8(q[u]));
          }
        }
      }
    } else if constexpr (RC > 0) {
      // all of a thread's loads are issued before its first store, so that
      // their latencies overlap
      constexpr int IHc = ST_TH + 2 * (RC + 3), IWc = ST_TW + 2 * (RC + 3);
      constexpr int NR = (IHc + ST_THREADS / 32 - 1) / (ST_THREADS / 32), NC = (IWc + 31) / 32;
      uint32_t v[NR][NC];
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        // rows and columns past the tile re-read its last row / column (every
        // address stays inside the tile's footprint); they are not stored
        const int iy = min(warp + k * (ST_THREADS / 32), IHc - 1);
        const int gy = interior ? y0 - HALO + iy : reflect101(y0 - HALO + iy, H);
        const Tin* row = img + (size_t)gy * W;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int ix = min(lane + 32 * c, IWc - 1);
          const int gx = interior ? x0 - HALO + ix : reflect101(x0 - HALO + ix, W);
          v[k][c] = (uint32_t)row[gx];
        }
      }
#pragma unroll
      for (int k = 0; k < NR; ++k) {
        const int iy = warp + k * (ST_THREADS / 32);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const int ix = lane + 32 * c;
          if (iy < IHc && ix < IWc) sI[iy * IW + coff + ix] = (uint16_t)v[k][c];
          vmax = max(vmax, v[k][c]);
        }
      }
    } else {
      for (int iy = warp; iy < IH; iy += ST_THREADS / 32) {
        const int gy = interior ? y0 - HALO + iy : reflect101(y0 - HALO + iy, H);
        const Tin* row = img + (size_t)gy * W;
        uint16_t* dst = sI + iy * IW + coff;
        for (int ix = lane; ix < IWn; ix += 32) {
          const int gx = interior ? x0 - HALO + ix : reflect101(x0 - HALO + ix, W);
          dst[ix] = (uint16_t)row[gx];
          vmax = max(vmax, (uint32_t)row[gx]);
        }
      }
    }
    if (sizeof(Tin) > 1) {
      vmax = __reduce_max_sync(0xffffffffu, vmax);
      if (lane == 0) atomicMax(&s_imax, vmax);
    }
  }
  __syncthreads();

  // Exact smoothing, L' = sum_i sum_j Q_i Q_j I, in u32 / u64.  A tile whose
  // inputs all lie in [0, narrow_max] keeps every horizontal sum below 2^31
  // and every vertical pair of them below 2^32.  A wider tile (16-bit data
  // above that) is smoothed twice, once for the high byte and once for the
  // low byte of each input, and L' = 2^8 L'(high) + L'(low); each part's sums
  // then stay below 2^28.
  const bool wide = sizeof(Tin) > 1 && s_imax > a.narrow_max;
  float lmax = 0.0f;
  // part 0: high bytes, 1: low bytes, 2: the inputs themselves; the last
  // part rounds L' to FP32.  The part is a compile-time constant of each
  // instance, so the narrow case extracts nothing.
  auto smooth = [&](auto part_c) {
  constexpr int part = decltype(part_c)::value;
  constexpr uint32_t shift = part == 0 ? 8u : 0u, mask = part == 1 ? 0xffu : 0xffffffffu;
  constexpr bool last = part != 0;

  // ---- B: horizontal Gaussian, exact u32 (sum Q_i I < 2^31)
  if constexpr (RC > 0) {
    // four adjacent outputs per thread from 2R + 4 inputs, stored as one
    // 16-byte vector; the lanes of a warp take neighbouring output quads of a
    // row.  The last quad's two outputs past ST_TW + 6 are not read later.
    constexpr int NW = 2 * RC + 4;
    constexpr int NQ = (ST_TW + 6 + 3) / 4;
    constexpr int CO = in_org(RC + 3) - (RC + 3);
    static_assert(4 * NQ <= P_STRIDE, "the horizontal pass's row holds every quad");
    for (int i = tid; i < IH * NQ; i += ST_THREADS) {
      const int iy = i / NQ, qq = i - iy * NQ;
      const uint16_t* row = sI + iy * IW + CO + 4 * qq;
      uint32_t w[NW];
#pragma unroll
      for (int k = 0; k < NW; ++k) w[k] = ((uint32_t)row[k] >> shift) & mask;
      uint32_t acc[4];
#pragma unroll
      for (int o = 0; o < 4; ++o) {
        acc[o] = (uint32_t)a.taps.q[RC] * w[RC + o];
#pragma unroll
        for (int j = 0; j < RC; ++j) acc[o] += (uint32_t)a.taps.q[j] * (w[j + o] + w[2 * RC - j + o]);
      }
      *reinterpret_cast<uint4*>(sP + iy * PWs + 4 * qq) = make_uint4(acc[0], acc[1], acc[2], acc[3]);
    }
  } else {
    const int coff = ORG - HALO;
    for (int i = tid; i < IH * PW; i += ST_THREADS) {
      int iy = i / PW, px = i - iy * PW;
      const uint16_t* row = sI + iy * IW + coff + px;
      uint32_t acc = (uint32_t)q[R] * (((uint32_t)row[R] >> shift) & mask);
      for (int j = 0; j < R; ++j)
        acc += (uint32_t)q[j] * ((((uint32_t)row[j] >> shift) & mask) + (((uint32_t)row[2 * R - j] >> shift) & mask));
      sP[iy * PWs + px] = acc;
    }
  }
  __syncthreads();

  // ---- C: vertical Gaussian, exact u64: L' = sum_i sum_j Q_i Q_j I
  //      (a pair Q_j (P_j + P_2R-j) of horizontal sums stays below 2^32);
  //      also L' rounded to FP32 and the tile's largest value of it
  if constexpr (RC > 0) {
    // C_RUN vertically adjacent outputs per thread from one window of
    // 2R + C_RUN horizontal sums; lanes take columns, and one pass covers the
    // tile.  The last run's rows past the tile read the horizontal pass's
    // spare rows (never written) and are not stored.
    constexpr int RUN = C_RUN, NW = 2 * RC + RUN;
    constexpr int NRUN = (ST_TH + 6 + RUN - 1) / RUN;
    for (int i = tid; i < NRUN * PW; i += ST_THREADS) {
      const int lr = i / PW, px = i - lr * PW;
      const int ly0 = RUN * lr;
      const uint32_t* col = sP + ly0 * PWs + px;
      uint32_t w[NW];
#pragma unroll
      for (int k = 0; k < NW; ++k) w[k] = col[k * PWs];
#pragma unroll
      for (int o = 0; o < RUN; ++o) {
        unsigned long long acc = (unsigned long long)(uint32_t)a.taps.q[RC] * w[RC + o];
#pragma unroll
        for (int j = 0; j < RC; ++j)
          acc += (unsigned long long)(uint32_t)a.taps.q[j] * (unsigned long long)(w[j + o] + w[2 * RC - j + o]);
        if (ly0 + o < LH) {
          const int idx = (ly0 + o) * PW + px;
          if constexpr (part == 1) acc += sL[idx] << 8;
          sL[idx] = acc;
          if constexpr (last) {
            const float fv = __ull2float_rn(acc);
            sLf[idx] = fv;
            lmax = fmaxf(lmax, fv);
          }
        }
      }
    }
  } else {
    for (int i = tid; i < LH * PW; i += ST_THREADS) {
      int ly = i / PW, px = i - ly * PW;
      const uint32_t* col = sP + ly * PWs + px;
      unsigned long long acc = (unsigned long long)(uint32_t)q[R] * col[R * PWs];
      for (int j = 0; j < R; ++j)
        acc += (unsigned long long)(uint32_t)q[j] * (unsigned long long)(col[j * PWs] + col[(2 * R - j) * PWs]);
      if constexpr (part == 1) acc += sL[i] << 8;
      sL[i] = acc;
      if constexpr (last) {
        const float fl = __ull2float_rn(acc);
        sLf[i] = fl;
        lmax = fmaxf(lmax, fl);
      }
    }
  }
  };
  if (wide) {
    smooth(std::integral_constant<int, 0>{});
    __syncthreads();  // the high part's vertical pass has read sP
    smooth(std::integral_constant<int, 1>{});
  } else {
    smooth(std::integral_constant<int, 2>{});
  }
  {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(lmax));
    if ((tid & 31) == 0) atomicMax(&s_lmax, m);
  }
  __syncthreads();

  // ---- D: FP32 Hessian (gradient) of the rounded L and FP32 k- with its
  //         error bound on the tile plus a one-pixel ring.  A thread takes a
  //         column strip of DRUN points: it forms the row filters s, d2 and
  //         d1 of the strip's DRUN + 4 rows (row_filters32) in registers and
  //         the column filters from them (hess32_v, grad32_v), and stores k-,
  //         its bound and the entries, which the direction test reads.
  // Bound on |fl(H) x fl(1/D) - H'/D| for each entry (hess32), u = 2^-24,
  // with 0 <= L' <= Lm (Lm: the tile's largest rounded L, >= L'(1 - u)).
  // Each rounding adds at most u |its result|, times the coefficient that
  // carries it to the entry.  With the ranges of the intermediates (e and
  // l1 + l3 in [0, 2Lm], s in [0, 16Lm], d2 in [-2Lm, 2Lm], d1 in
  // [-3Lm, 3Lm]) the sum is, for Lxx, 64 (conversion) + 16 x 4 (row
  // filters) + 72 (column filter) + 2 x 64 (scaling) = 328 u Lm / D; for
  // Lyy 64 + 4 x 36 + 64 + 128 = 400; for Lxy 36 + 6 x 6 + 36 + 72 = 180.
  // delta = 448 u Lm / D, rounded up, covers all three with room for the
  // second-order terms.
  // Directed edges: Gx 96 (conversion) + 16 x 6 (row filters) + 108 (column
  // filter) + 96 (scaling) = 396 u Lm / D, Gy 96 + 6 x 36 + 96 + 96 = 504;
  // delta = 576 u Lm / D.
  const float delta = __fmul_ru(__fmul_ru(__uint_as_float(s_lmax), a.invD), EDGE ? 0x1.2p-15f : 0x1.cp-16f);
  {
    constexpr int DRUN = 5;
    constexpr int NSTRIP = (ST_TH + 2 + DRUN - 1) / DRUN;
    for (int t = tid; t < NSTRIP * HW2; t += ST_THREADS) {
      const int strip = t / HW2, hx = t - strip * HW2;
      const int hy0 = strip * DRUN;
      float rs[DRUN + 4], rd2[DRUN + 4], rd1[DRUN + 4];
#pragma unroll
      for (int r = 0; r < DRUN + 4; ++r) {
        // rows past the tile's last point repeat its last row (not used)
        const int ly = min(hy0 + r, LH - 1);
        row_filters32(sLf + ly * PW + hx, rs[r], rd2[r], rd1[r]);
        if (r < 4) continue;
        const int o = r - 4;
        if (hy0 + o >= HH2) continue;
        const int i = (hy0 + o) * HW2 + hx;
        if constexpr (EDGE) {
          float gx, gy;
          grad32_v(rd1[o], rd1[o + 1], rd1[o + 2], rd1[o + 3], rd1[o + 4], rs[o], rs[o + 1], rs[o + 3], rs[o + 4],
                   a.invD, gx, gy);
          const float g = __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
          sK[i] = -g;
          // |grad| is 1-Lipschitz: the inputs move it by <= sqrt 2 delta; four
          // roundings by <= 4 u |grad|
          sE[i] = __fmaf_ru(1.5f, delta, 4.0f * U32 * g);
          sHa[i] = gx;
          sHb[i] = gy;
        } else {
          float fa, fb, fc;
          hess32_v(rd2[o], rd2[o + 1], rd2[o + 2], rd2[o + 3], rd2[o + 4], rs[o], rs[o + 2], rs[o + 4], rd1[o],
                   rd1[o + 1], rd1[o + 3], rd1[o + 4], a.invD, fa, fb, fc);
          float k, ek, hdf, rad;
          eig32_k(fa, fb, fc, k, ek, hdf, rad);
          sK[i] = k;
          // an eigenvalue moves by at most the spectral norm of the
          // perturbation, which is at most its Frobenius norm, <= 2 delta
          sE[i] = __fmaf_ru(3.0f, delta, ek);
          sHa[i] = fa;
          sHb[i] = fb;
          sHc[i] = fc;
        }
      }
    }
  }
  __syncthreads();

  // ---- E1: threshold test of the tile's pixels, 4 per thread: certainly no
  //          ridge, undecided (listed for the exact test), or a candidate for
  //          the direction test (listed, so that E2 runs it with full warps:
  //          candidates cluster along the ridges)
  uint16_t* sC = sR;  // the candidate list; the ridge list takes these bytes after the exact test
  {
    const int lane = tid & 31;
    unsigned m[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int pi = tid + j * ST_THREADS;
      const int ty = pi / ST_TW, tx = pi - ty * ST_TW;
      const int gx = x0 + tx, gy = y0 + ty;
      uint8_t verdict = 0;
      bool cand = false;
      if (gx < W && gy < H) {
        const int c = (ty + 1) * HW2 + tx + 1;
        const float dk = sK[c] - a.tau;  // exact near the boundary (Sterbenz)
        const float ek = sE[c];
        if (dk >= ek) {
          verdict = 0;
        } else if (!(dk < -ek)) {
          verdict = 2;
          const int k = atomicAdd(&s_nu, 1);
          if (RD_GUARD(k < ST_TW * ST_TH, a.stats)) sU[k] = (uint16_t)pi;
        } else {
          cand = true;
        }
      }
      sV[pi] = verdict;
      m[j] = __ballot_sync(0xffffffffu, cand);
    }
    // one list reservation per warp for its four rows of candidates
    const int n = __popc(m[0]) + __popc(m[1]) + __popc(m[2]) + __popc(m[3]);
    if (n) {
      int base = 0;
      if (lane == 0) base = atomicAdd(&s_ncand, n);
      base = __shfl_sync(0xffffffffu, base, 0);
      const unsigned below = (1u << lane) - 1u;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = base + __popc(m[j] & below);
        if (((m[j] >> lane) & 1u) && RD_GUARD(k < ST_TW * ST_TH, a.stats))
          sC[k] = (uint16_t)(tid + j * ST_THREADS);
        base += __popc(m[j]);
      }
    }
  }
  __syncthreads();
  // ---- E2: direction test of the candidates (k- certainly below tau):
  //          X- with its bound, then the certified local-minimum test
  {
    const int ncand = s_ncand;
    for (int t = tid; t < ncand; t += ST_THREADS) {
      const int pi = sC[t];
      const int ty = pi / ST_TW, tx = pi - ty * ST_TW;
      const int gx = x0 + tx, gy = y0 + ty;
      const int hy = ty + 1, hx = tx + 1, c = hy * HW2 + hx;
      const float k = sK[c], ek = sE[c];
      float X, Y, eX;
      bool dir_ok;
      if constexpr (EDGE) {
        // unit gradient: (Gx, Gy) moves by <= sqrt 2 delta, so X by <=
        // 2 sqrt 2 delta / |grad| plus the roundings
        const float gxf = sHa[c], gyf = sHb[c];
        const float g = -k;
        dir_ok = g > 4.0f * delta && g > 0.0f;
        X = __fdiv_rn(gxf, g);
        Y = __fdiv_rn(gyf, g);
        if (X < 0.0f || (X == 0.0f && Y < 0.0f)) {
          X = -X;
          Y = -Y;
        }
        eX = 3.0f * delta / (g - 2.0f * delta) + 4.0f * U32;
      } else {
        const float fa = sHa[c], fb = sHb[c], fc = sHc[c];
        float k2, ek2, hdf, rad;
        eig32_k(fa, fb, fc, k2, ek2, hdf, rad);
        float M = fabsf(fa) + fabsf(fb) + fabsf(fc);
        if (gx == 0 || gx == W - 1 || gy == 0 || gy == H - 1) {
          // On a border row or column the reflect-101 extension of L' is
          // symmetric about that line, so the exact Hxy' is 0 and X- is an
          // exact axis: (1, 0) where Lxx < Lyy, (0, 1) where Lxx > Lyy (the
          // other candidate vector is only rounding).  hdf is within delta
          // (plus a relative 2^-24) of (Lxx - Lyy) / 2, so |hdf| > 2 delta
          // fixes the sign, and the sample offsets are exact integers.
          dir_ok = fabsf(hdf) > 2.0f * delta;
          X = hdf < 0.0f ? 1.0f : 0.0f;
          Y = 1.0f - X;
          eX = 0.0f;
        } else {
          dir_ok = eig32_dir(fb, hdf, rad, M, delta, X, Y, eX);
        }
      }
      const int verdict = dir_ok ? ridge_fast(sK, sE, HW2, hy, hx, gx, gy, H, W, k, ek, a.tau, X, Y, eX) : 2;
      sV[pi] = (uint8_t)verdict;
      if (verdict == 2) {
        const int k = atomicAdd(&s_nu, 1);
        if (RD_GUARD(k < ST_TW * ST_TH, a.stats)) sU[k] = (uint16_t)pi;
      }
    }
  }
  __syncthreads();
  if (tid == 0 && s_nu) atomicAdd(&a.stats->fallbacks, (unsigned long long)s_nu);
  {
    // exact test of the listed pixels, FB_CHUNK at a time: first one thread
    // per (pixel, neighbour) for the exact k- of the 3x3 neighbourhood (the
    // bilinear corners of both samples lie in it) and the centre's X-, then
    // one thread per pixel for the decision.  The FP32 entries are dead now.
    double* sKn = reinterpret_cast<double*>(smem + Ls.x);  // FB_CHUNK x 9
    double* sXc = sKn + FB_CHUNK * 9;                      // FB_CHUNK x 2
    uint8_t* sDg = reinterpret_cast<uint8_t*>(sXc + FB_CHUNK * 2);
    const int nu = s_nu;
    for (int c0 = 0; c0 < nu; c0 += FB_CHUNK) {
      const int nc = min(FB_CHUNK, nu - c0);
      for (int t = tid; t < nc * 9; t += ST_THREADS) {
        const int p = t / 9, n = t - p * 9;
        const int pi = sU[c0 + p];
        const int ty = pi / ST_TW, tx = pi - ty * ST_TW;
        if constexpr (EDGE) {
          long long gxi, gyi;
          grad_exact(sL, PW, ty + n / 3, tx + n % 3, gxi, gyi);
          const Grad64 e = grad64(gxi, gyi, a.D64, -a.tau64);
          sKn[t] = -e.g;
          if (n == 4) {
            sXc[2 * p] = e.X;
            sXc[2 * p + 1] = e.Y;
            sDg[p] = (e.X == 0.0 && e.Y == 0.0) ? 1 : 0;
          }
        } else {
          long long ha, hc, hb;
          hess_exact(sL, PW, ty + n / 3, tx + n % 3, ha, hc, hb);
          double ea, ec, eb;
          const double k = eigen64_k(ha, hc, hb, a.D64, ea, ec, eb);  // all nine lanes together
          sKn[t] = k;
          if (n == 4) {  // the centre's X- too
            Eig64 e;
            eigen64_dir(ea, ec, eb, k, e);
            sXc[2 * p] = e.X;
            sXc[2 * p + 1] = e.Y;
            sDg[p] = e.degenerate ? 1 : 0;
          }
        }
      }
      __syncthreads();
      for (int p = tid; p < nc; p += ST_THREADS) {
        const int pi = sU[c0 + p];
        const int ty = pi / ST_TW, tx = pi - ty * ST_TW;
        sV[pi] = ridge_exact_nb(sKn + 9 * p, sXc[2 * p], sXc[2 * p + 1], sDg[p] != 0, x0 + tx, y0 + ty, H, W,
                                a.tau64)
                     ? 1
                     : 0;
      }
      __syncthreads();
    }
  }
  // every verdict is now 0 or 1: flags holds pixel j's in bit 2j
  int flags = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) flags |= (int)sV[tid + j * ST_THREADS] << (2 * j);

  // ---- compaction: one block-wide exclusive scan of the per-thread counts
  //      into a list of the tile's ridge pixels (record order inside a tile
  //      is immaterial downstream: the fit's annulus sums are exact integers)
  const int lane = tid & 31, warp = tid >> 5;
  const int mine = __popc(flags & 0x55);  // every verdict is now 0 or 1
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) sScan[warp] = incl;
  __syncthreads();
  int wpre = 0, base = 0;
  for (int w = 0; w < ST_THREADS / 32; ++w) {
    const int c = sScan[w];
    wpre += (w < warp) ? c : 0;
    base += c;
  }
  {
    int p0 = wpre + incl - mine;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((flags >> (2 * j)) & 1) sR[p0++] = (uint16_t)(tid + j * ST_THREADS);
  }
  const int total = base;
  const int tile = blockIdx.y * a.rl.n_stx + blockIdx.x;
  const size_t tbase = (size_t)f * a.rl.n_stx * a.rl.n_sty + tile;
  if (tid == 0) {
    int start = total ? atomicAdd(&a.rl.count[f], total) : 0;
    sScan[ST_THREADS / 32] = start;
    int keep = max(0, min(total, a.rl.cap - start));
    if (keep < total) atomicOr(&a.stats->overflow, 1);
    a.rl.tile_off[tbase] = total ? start : 0;
    a.rl.tile_cnt[tbase] = keep;
    if (total) atomicAdd(&a.stats->ridge, (unsigned long long)total);
  }
  __syncthreads();
  // ---- records: the pixel and its exact Hessian (ridges) or exact direction
  //      (edges), list entries over threads
  const int start = sScan[ST_THREADS / 32];
  const int keep = max(0, min(total, a.rl.cap - start));
  for (int t = tid; t < keep; t += ST_THREADS) {
    const int pi = sR[t];
    const int ty = pi / ST_TW, tx = pi - ty * ST_TW;
    const size_t g = (size_t)f * a.rl.cap + start + t;
    a.rl.xy[g] = (uint32_t)(x0 + tx) | ((uint32_t)(y0 + ty) << 16);
    if constexpr (EDGE) {
      long long gxi, gyi;
      grad_exact(sL, PW, ty + 1, tx + 1, gxi, gyi);
      const Grad64 e = grad64(gxi, gyi, a.D64, -a.tau64);
      // the double direction as a float pair (|X - (hi + lo)| <= 2^-49) and
      // the vote-rounding margins of an exact direction
      const float xh = __double2float_rn(e.X), yh = __double2float_rn(e.Y);
      const float xl = __double2float_rn(e.X - (double)xh), yl = __double2float_rn(e.Y - (double)yh);
      const float eXr = 7.105427e-15f;  // 2^-47
      a.rl.dir[g] = make_float4(xh, yh, xl, yl);
      a.rl.kvote[g] = make_float2(1.25f * (fmaxf(fabsf(xl), fabsf(yl)) + eXr + U32) + U32, 1.25f * eXr + 2.842171e-14f);
      a.rl.hess[3 * g + 0] = 0;
      a.rl.hess[3 * g + 1] = 0;
      a.rl.hess[3 * g + 2] = 0;
      a.rl.x64[g] = make_double2(e.X, e.Y);
    } else {
      long long hxx, hyy, hxy;
      hess_exact(sL, PW, ty + 1, tx + 1, hxx, hyy, hxy);
      a.rl.hess[3 * g + 0] = hxx;
      a.rl.hess[3 * g + 1] = hyy;
      a.rl.hess[3 * g + 2] = hxy;
    }
  }
}

// K2: X- of each ridge pixel as a double-float from its exact Hessian, and
// the vote-rounding margins.  With P = Hxx' - Hyy', Bq = 2 Hxy',
// R = sqrt(P^2 + Bq^2): X- is proportional to (Bq, -(P + R)) for P >= 0 and
// to (-(|P| + R), Bq) otherwise; both components are computed without
// cancellation, so the direction is accurate to ~2^-44.
__global__ void __launch_bounds__(256) k_ridge_refine(RidgeList rl) {
  const int gstride = gridDim.x * blockDim.x;
  {
    const int f = blockIdx.y;  // one grid row per frame
    int cnt = min(rl.count[f], rl.cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gstride) {
      size_t g = (size_t)f * rl.cap + i;
      long long A = rl.hess[3 * g + 0], C = rl.hess[3 * g + 1], B = rl.hess[3 * g + 2];
      long long P = A - C, Bq = 2 * B;
      dfl dP = df_from_ll(P), dB = df_from_ll(Bq);
      dfl Rr = df_sqrt(df_add(df_mul(dP, dP), df_mul(dB, dB)));
      dfl aP = P >= 0 ? dP : dfl{-dP.hi, -dP.lo};
      dfl Wc = df_add(aP, Rr);
      dfl vx, vy;
      if (P >= 0) {
        vx = dB;
        vy = {-Wc.hi, -Wc.lo};
      } else {
        vx = {-Wc.hi, -Wc.lo};
        vy = dB;
      }
      dfl nrm = df_sqrt(df_add(df_mul(vx, vx), df_mul(vy, vy)));
      dfl X = df_div(vx, nrm), Y = df_div(vy, nrm);
      if (X.hi < 0.0f || (X.hi == 0.0f && Y.hi < 0.0f)) {
        X = {-X.hi, -X.lo};
        Y = {-Y.hi, -Y.lo};
      }
      // bounds: double-float direction error <= 2^-40; the double-precision
      // definition's own error <= 2^-48 * cond, cond = |H| / |v| (its
      // eigenvector formula cancels when the eigenvalue gap is small)
      float M = fabsf(__ll2float_rn(A)) + fabsf(__ll2float_rn(B)) + fabsf(__ll2float_rn(C));
      float cond = 2.0f * M / fmaxf(nrm.hi, 1e-30f);
      float eXr = 9.094947e-13f + 3.5527137e-15f * cond;  // 2^-40 + 2^-48 cond
      float lo = fmaxf(fabsf(X.lo), fabsf(Y.lo));
      float kfast = 1.25f * (lo + eXr + U32) + U32;
      float kref = 1.25f * eXr + 2.842171e-14f;           // + 2^-45
      rl.dir[g] = make_float4(X.hi, Y.hi, X.lo, Y.lo);
      rl.kvote[g] = make_float2(kfast, kref);
    }
  }
}

size_t stencil_smem_bytes(int R) { return stencil_smem_layout(R).total; }

// Gaussian half-width compiled in: R = ceil(4 sigma) = 8 for sigma in (1.75, 2]
constexpr int ST_RC = 8;

template <typename Tin, int RC, bool EDGE>
static void launch_stencil_t(const StencilArgs& a, dim3 grid, size_t sm, cudaStream_t st) {
  cudaFuncSetAttribute(k_stencil_ridge<Tin, RC, EDGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_stencil_ridge<Tin, RC, EDGE><<<grid, ST_THREADS, sm, st>>>(a);
}

template <typename Tin, bool EDGE>
static void launch_stencil_r(const StencilArgs& a, dim3 grid, size_t sm, cudaStream_t st) {
  if (a.taps.R == ST_RC)
    launch_stencil_t<Tin, ST_RC, EDGE>(a, grid, sm, st);
  else
    launch_stencil_t<Tin, 0, EDGE>(a, grid, sm, st);
}


cudaError_t launch_stencil(const StencilArgs& args, int dtype, cudaStream_t st) {
  StencilArgs a = args;
  long long S = 0;
  for (int i = 0; i <= 2 * a.taps.R; ++i) S += a.taps.q[i];
  a.narrow_max = (uint32_t)((4294967295LL) / (2 * S));
  const size_t px_bytes = dtype == 0 ? 1 : 2;
  a.vec_rows = ((uintptr_t)a.frames % 16 == 0) && ((size_t)a.W * px_bytes % 16 == 0) ? 1 : 0;
  dim3 grid((a.W + ST_TW - 1) / ST_TW, (a.H + ST_TH - 1) / ST_TH, a.n);
  size_t sm = stencil_smem_bytes(a.taps.R);
  if (dtype == 0)
    a.edge ? launch_stencil_r<uint8_t, true>(a, grid, sm, st) : launch_stencil_r<uint8_t, false>(a, grid, sm, st);
  else
    a.edge ? launch_stencil_r<uint16_t, true>(a, grid, sm, st) : launch_stencil_r<uint16_t, false>(a, grid, sm, st);
  return cudaGetLastError();
}

cudaError_t launch_refine(const RidgeList& rl, int n_frames, int n_sm, cudaStream_t st) {
  const dim3 grid((unsigned)max(1, (n_sm * 4 + n_frames - 1) / n_frames), (unsigned)n_frames);
  k_ridge_refine<<<grid, 256, 0, st>>>(rl);
  return cudaGetLastError();
}

}  // namespace rd
