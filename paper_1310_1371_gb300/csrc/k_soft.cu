// k_soft.cu -- the differentiable (soft) ring score, its gradients with
// respect to the ring parameters and to the image, and gradient-ascent
// refinement of rings.
//
// The paper has no differentiable form.  The score extends its voting and
// scoring steps (Results, "Directed ridge detection & votes collection",
// "Local maxima detection in a noisy parameter space") smoothly:
//   Score(c, rho) = (1/rho) sum_{p in ridge} m(p) a(p) sum_{s=+-1} sum_{q in corners(v)}
//                   bil(v, q) exp(-|q - c|^2 / (2 sigma(rho)^2)),
//   v = p + s rho X(p),  m(p) = logistic((tau - k(p)) / T),  T = |tau| / 4,
//   a(p) = exp(-(|p - c| - rho)^2 / (2 sa^2)),  sa = w / 2,
// with the hard directed-ridge set of the frame held fixed, grid points
// outside the image receiving nothing, and sigma(rho) = sig_a rho + sig_b.
// a(p) is the ring's soft annulus (Results, "Ridge points classification &
// sub-pixel accuracy": the ridge pixels within an annulus of half-width w
// around a ring are its own): it keeps pixels of neighbouring rings, which
// lie off the circle, out of the score.
// The image gradient flows through k and X to the exact-arithmetic chain
// eigen <- 5x5 second-order Sobel / 64 <- Gaussian, each stencil with
// reflect-101 borders; its adjoint is applied as gathers, recomputing the
// stencil stage instead of storing per-ring state.  Everything is FP64.
#include "rd_internal.cuh"
#include "rd_cert.cuh"

#include <cmath>

namespace rd {

__device__ __forceinline__ int refl101(int i, int n) {
  i = i < 0 ? -i : i;
  return i >= n ? 2 * (n - 1) - i : i;
}

template <typename T>
__device__ __forceinline__ double pix(const void* frames, size_t i) {
  return (double)reinterpret_cast<const T*>(frames)[i];
}

// ---- S1/S2: separable Gaussian (taps Q_i / S) ---------------------------------
template <typename T>
__global__ void k_soft_hpass(SoftArgs a) {
  const size_t total = (size_t)a.n * a.H * a.W;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t row = i / a.W;
    const int x = (int)(i - row * a.W);
    const size_t base = row * a.W;
    double s = 0.0;
    for (int t = -a.R; t <= a.R; ++t) s += a.g[t + a.R] * pix<T>(a.frames, base + refl101(x + t, a.W));
    a.t0[i] = s;
  }
}

__global__ void k_soft_vpass(SoftArgs a) {
  const size_t plane = (size_t)a.H * a.W, total = plane * a.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t f = i / plane;
    const size_t r = i - f * plane;
    const int y = (int)(r / a.W), x = (int)(r - (size_t)y * a.W);
    const double* src = a.t0 + f * plane + x;
    double s = 0.0;
    for (int t = -a.R; t <= a.R; ++t) s += a.g[t + a.R] * src[(size_t)refl101(y + t, a.H) * a.W];
    a.t1[i] = s;
  }
}

__constant__ double c_s5[5] = {1, 4, 6, 4, 1};
__constant__ double c_d1[5] = {-1, -2, 0, 2, 1};
__constant__ double c_d2[5] = {1, 0, -2, 0, 1};

// eigen step (O3) in the oracle's operation order
struct SoftEig {
  double k, X, Y;
  bool degenerate, use1, flip;
};
__device__ __forceinline__ SoftEig soft_eigen(double a, double c, double b) {
  SoftEig e;
  const double half_tr = d_mul(d_add(a, c), 0.5);
  const double half_df = d_mul(d_sub(a, c), 0.5);
  const double rad = d_sqrt(d_add(d_mul(half_df, half_df), d_mul(b, b)));
  e.k = d_sub(half_tr, rad);
  const double v1x = b, v1y = d_sub(e.k, a), v2x = d_sub(e.k, c), v2y = b;
  const double n1 = d_add(d_mul(v1x, v1x), d_mul(v1y, v1y));
  const double n2 = d_add(d_mul(v2x, v2x), d_mul(v2y, v2y));
  e.use1 = n1 >= n2;
  const double vx = e.use1 ? v1x : v2x, vy = e.use1 ? v1y : v2y, nn = e.use1 ? n1 : n2;
  e.degenerate = nn == 0.0;
  e.X = 0.0;
  e.Y = 0.0;
  e.flip = false;
  if (!e.degenerate) {
    const double nrm = d_sqrt(nn);
    double X = d_div(vx, nrm), Y = d_div(vy, nrm);
    e.flip = X < 0.0 || (X == 0.0 && Y < 0.0);
    e.X = e.flip ? -X : X;
    e.Y = e.flip ? -Y : Y;
  }
  return e;
}

// ---- S3/S4: Hessian, k- and X- (O2-O3), directed-ridge mask (O4) and ridge
// records, one CTA per 32 x 32 tile.  Every pixel is tested in FP32 with a
// certified bound (the detector's stencil-stage arithmetic, rd_cert.cuh)
// from the rounded FP64 L; the few pixels it cannot decide, and the records,
// get the FP64 Hessian and eigen step of the definition.  Records of a tile
// are contiguous (order inside a tile unspecified), so that the score can
// visit only the tiles near a ring.
constexpr int SOFT_T = 32;
constexpr int SOFT_PW = SOFT_T + 6;  // L rows and columns of a tile: the Hessian ring + the 5x5 stencil
constexpr int SOFT_HW = SOFT_T + 2;  // Hessian tile: the pixels and a one-pixel ring
constexpr int SOFT_FB = 256 / 9;     // pixels per step of the exact test (9 threads each)

// FP64 Hessian of L at Hessian-tile coordinates (hy, hx) (rows hy .. hy + 4
// and columns hx .. hx + 4 of the L tile, reflect-101 already applied): the
// 5x5 second-order Sobel / 64.
__device__ __forceinline__ void soft_hess64(const double* sLd, int hy, int hx, double& A, double& C, double& B) {
  double hxx = 0.0, hyy = 0.0, hxy = 0.0;
  for (int dy = 0; dy < 5; ++dy) {
    const double* row = sLd + (hy + dy) * SOFT_PW + hx;
    double sx = 0.0, d2x = 0.0, d1x = 0.0;
    for (int dx = 0; dx < 5; ++dx) {
      const double l = row[dx];
      sx += c_s5[dx] * l;
      d2x += c_d2[dx] * l;
      d1x += c_d1[dx] * l;
    }
    hxx += c_s5[dy] * d2x;
    hyy += c_d2[dy] * sx;
    hxy += c_d1[dy] * d1x;
  }
  A = hxx / 64.0;
  C = hyy / 64.0;
  B = hxy / 64.0;
}

// reflect-101 with far indices (only for discarded outputs of partial tiles) clamped
__device__ __forceinline__ int refl101c(int i, int n) {
  i = i < 0 ? -i : i;
  i = i >= n ? 2 * (n - 1) - i : i;
  return min(max(i, 0), n - 1);
}

__global__ void __launch_bounds__(256) k_soft_mask(SoftArgs a) {
  __shared__ double sLd[SOFT_PW * SOFT_PW];                 // FP64 L of the tile
  __shared__ float sLf[SOFT_PW * SOFT_PW];                  // rounded to FP32
  __shared__ __align__(16) unsigned char sRow[3 * SOFT_PW * SOFT_HW * 4];  // row filters; later the exact test's scratch
  __shared__ float sK[SOFT_HW * SOFT_HW], sE[SOFT_HW * SOFT_HW];
  __shared__ uint16_t sU[SOFT_T * SOFT_T], sR[SOFT_T * SOFT_T];
  __shared__ uint8_t sV[SOFT_T * SOFT_T];
  __shared__ int s_warp[8], s_start, s_nu;
  __shared__ unsigned s_lmax;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int f = blockIdx.z, x0 = blockIdx.x * SOFT_T, y0 = blockIdx.y * SOFT_T;
  const int H = a.H, W = a.W;
  const size_t plane = (size_t)H * W;
  const double* L = a.t1 + (size_t)f * plane;
  if (tid == 0) {
    s_nu = 0;
    s_lmax = 0u;
  }
  __syncthreads();
  // L of the tile with a 3-pixel ring (reflect-101 at the frame's borders)
  float lmax = 0.0f;
  for (int i = tid; i < SOFT_PW * SOFT_PW; i += 256) {
    const int iy = i / SOFT_PW, ix = i - iy * SOFT_PW;
    const double v = L[(size_t)refl101c(y0 - 3 + iy, H) * W + refl101c(x0 - 3 + ix, W)];
    sLd[i] = v;
    const float fv = __double2float_rn(v);
    sLf[i] = fv;
    lmax = fmaxf(lmax, fabsf(fv));
  }
  {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(lmax));
    if (lane == 0) atomicMax(&s_lmax, m);
  }
  __syncthreads();
  // FP32 row filters s, d2, d1 of every L row, at the Hessian tile's columns
  float* sRs = reinterpret_cast<float*>(sRow);
  float* sRd2 = sRs + SOFT_PW * SOFT_HW;
  float* sRd1 = sRd2 + SOFT_PW * SOFT_HW;
  for (int i = tid; i < SOFT_PW * SOFT_HW; i += 256) {
    const int ly = i / SOFT_HW, hx = i - ly * SOFT_HW;
    const float* row = sLf + ly * SOFT_PW + hx;
    const float l0 = row[0], l1 = row[1], l2 = row[2], l3 = row[3], l4 = row[4];
    const float e = __fadd_rn(l0, l4);
    sRs[i] = __fmaf_rn(6.0f, l2, __fmaf_rn(4.0f, __fadd_rn(l1, l3), e));
    sRd2[i] = __fmaf_rn(-2.0f, l2, e);
    sRd1[i] = __fmaf_rn(2.0f, __fsub_rn(l3, l1), __fsub_rn(l4, l0));
  }
  // The detector's bound (hess32) for |L| <= Lm of either sign: each
  // rounding adds at most u |its result| times the coefficient that carries
  // it to the entry; with |e|, |l1 + l3| <= 2 Lm, |s| <= 16 Lm, |d2| <= 4 Lm,
  // |d1| <= 6 Lm and an exact scaling by 1/64 the sums are 304 (Lxx, Lyy) and
  // 180 (Lxy) u Lm / 64; delta = 512 u Lm / 64 = 2^-21 Lm.
  const float delta = __fmul_ru(__uint_as_float(s_lmax), 0x1p-21f);
  __syncthreads();
  for (int i = tid; i < SOFT_HW * SOFT_HW; i += 256) {
    float fa, fb, fc, k, ek, hdf, rad;
    hess32(sRs, sRd2, sRd1, SOFT_HW, i, 0.015625f, fa, fb, fc);
    eig32_k(fa, fb, fc, k, ek, hdf, rad);
    sK[i] = k;
    sE[i] = __fmaf_ru(3.0f, delta, ek);
  }
  __syncthreads();
  // certified test of the tile's pixels, 4 per thread; undecided ones to a list
  const float tau = (float)a.tau;
  int flags = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int pi = tid + 256 * j, ty = pi >> 5, tx = pi & 31, gx = x0 + tx, gy = y0 + ty;
    int verdict = 0;
    if (gx < W && gy < H) {
      const int hy = ty + 1, hx = tx + 1, c = hy * SOFT_HW + hx;
      const float k = sK[c], ek = sE[c], dk = k - tau;
      if (dk >= ek) {
        verdict = 0;
      } else if (!(dk < -ek)) {
        verdict = 2;
      } else {
        float fa, fb, fc, k2, ek2, hdf, rad, X, Y, eX;
        hess32(sRs, sRd2, sRd1, SOFT_HW, c, 0.015625f, fa, fb, fc);
        eig32_k(fa, fb, fc, k2, ek2, hdf, rad);
        const float M = fabsf(fa) + fabsf(fb) + fabsf(fc);
        verdict = eig32_dir(fb, hdf, rad, M, delta, X, Y, eX)
                      ? ridge_fast(sK, sE, SOFT_HW, hy, hx, gx, gy, H, W, k, ek, tau, X, Y, eX)
                      : 2;
      }
      if (verdict == 2) sU[atomicAdd(&s_nu, 1)] = (uint16_t)pi;
    }
    flags |= verdict << (2 * j);
  }
  __syncthreads();
  {
    // exact test: one thread per (pixel, neighbour) for the FP64 k- of the
    // 3x3 neighbourhood and the centre's X-, then one thread per pixel
    double* sKn = reinterpret_cast<double*>(sRow);  // SOFT_FB x 9
    double* sXc = sKn + SOFT_FB * 9;                // SOFT_FB x 2
    uint8_t* sDg = reinterpret_cast<uint8_t*>(sXc + SOFT_FB * 2);
    const int nu = s_nu;
    for (int c0 = 0; c0 < nu; c0 += SOFT_FB) {
      const int nc = min(SOFT_FB, nu - c0);
      for (int t = tid; t < nc * 9; t += 256) {
        const int p = t / 9, n = t - p * 9, pi = sU[c0 + p], ty = pi >> 5, tx = pi & 31;
        double A, C, B;
        soft_hess64(sLd, ty + n / 3, tx + n % 3, A, C, B);
        const SoftEig e = soft_eigen(A, C, B);
        sKn[t] = e.k;
        if (n == 4) {
          sXc[2 * p] = e.X;
          sXc[2 * p + 1] = e.Y;
          sDg[p] = e.degenerate ? 1 : 0;
        }
      }
      __syncthreads();
      for (int p = tid; p < nc; p += 256) {
        const int pi = sU[c0 + p], ty = pi >> 5, tx = pi & 31;
        sV[pi] = ridge_exact_nb(sKn + 9 * p, sXc[2 * p], sXc[2 * p + 1], sDg[p] != 0, x0 + tx, y0 + ty, H, W, a.tau)
                     ? 1
                     : 0;
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (((flags >> (2 * j)) & 3) == 2) flags ^= (2 ^ (int)sV[tid + 256 * j]) << (2 * j);
  // compaction: block-wide scan of the per-thread counts into the pixel list
  const int mine = __popc(flags & 0x55);
  int incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  int pre = 0, total = 0;
  for (int w = 0; w < 8; ++w) {
    pre += w < warp ? s_warp[w] : 0;
    total += s_warp[w];
  }
  {
    int p0 = pre + incl - mine;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if ((flags >> (2 * j)) & 1) sR[p0++] = (uint16_t)(tid + 256 * j);
  }
  const size_t t = ((size_t)f * a.n_ty + blockIdx.y) * a.n_tx + blockIdx.x;
  if (tid == 0) {
    const int start = total ? atomicAdd(&a.count[f], total) : 0;
    s_start = start;
    a.tile_off[t] = start;
    a.tile_cnt[t] = max(0, min(total, a.cap - start));
  }
  __syncthreads();
  // records: the FP64 Hessian, k-, X- and the soft mask weight
  const int start = s_start, keep = max(0, min(total, a.cap - start));
  for (int q = tid; q < keep; q += 256) {
    const int pi = sR[q], ty = pi >> 5, tx = pi & 31;
    double A, C, B;
    soft_hess64(sLd, ty + 1, tx + 1, A, C, B);
    const SoftEig e = soft_eigen(A, C, B);
    const size_t g = (size_t)f * a.cap + start + q;
    a.xy[g] = (uint32_t)(x0 + tx) | ((uint32_t)(y0 + ty) << 16);
    a.flags[g] = (uint8_t)((e.use1 ? 1 : 0) | (e.flip ? 2 : 0));
    a.rk[g] = e.k;
    a.rX[g] = e.X;
    a.rY[g] = e.Y;
    a.ra[g] = A;
    a.rb[g] = B;
    a.rc[g] = C;
    a.rm[g] = 1.0 / (1.0 + exp(-(a.tau - e.k) / a.temp));
  }
}

cudaError_t launch_soft_stencil(const SoftArgs& a, cudaStream_t st) {
  const unsigned grid = 152 * 8;
  if (a.dtype == RD_U8)
    k_soft_hpass<uint8_t><<<grid, 256, 0, st>>>(a);
  else if (a.dtype == RD_U16)
    k_soft_hpass<uint16_t><<<grid, 256, 0, st>>>(a);
  else
    k_soft_hpass<float><<<grid, 256, 0, st>>>(a);
  k_soft_vpass<<<grid, 256, 0, st>>>(a);
  k_soft_mask<<<dim3(a.n_tx, a.n_ty, a.n), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---- S5: score and gradients per ring -------------------------------------------
// exclusive prefix of the per-frame ring counts (one CTA)
__global__ void k_soft_offsets(const int* counts, int n, int* off) {
  __shared__ int part[1024];
  const int tid = threadIdx.x;
  const int per = (n + 1023) / 1024;
  int s = 0;
  for (int i = tid * per; i < min(n, (tid + 1) * per); ++i) s += max(counts[i], 0);
  part[tid] = s;
  __syncthreads();
  if (tid == 0) {
    int acc = 0;
    for (int t = 0; t < 1024; ++t) {
      const int v = part[t];
      part[t] = acc;
      acc += v;
    }
    off[n] = acc;
  }
  __syncthreads();
  int acc = part[tid];
  for (int i = tid * per; i < min(n, (tid + 1) * per); ++i) {
    off[i] = acc;
    acc += max(counts[i], 0);
  }
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;  // valid in thread 0
}

constexpr int SOFT_MAX_TILES = 256;  // tiles a ring visits through the tile index

// exp(x) for the score's Gaussian factors (x <= 0) in FP32: expf is within
// 2 ulp (relative 2.4e-7) and rounding x to FP32 moves it by at most
// 2^-24 |x|, so a factor with |x| <= 40.5 errs by under 3e-6 of itself;
// smaller factors (below e^-40.5) change a score by less than 1e-12 of its
// value whatever their error.  A score, a sum of positive factors, thus errs
// by under 3e-6 of its value.  The GB300's FP32 exponential runs at many
// times the rate of its FP64 one.
__device__ __forceinline__ double score_exp(double x) { return (double)expf((float)x); }

__global__ void __launch_bounds__(256) k_soft_score(SoftArgs a) {
  __shared__ double red[8];
  __shared__ int s_off[SOFT_MAX_TILES], s_pre[SOFT_MAX_TILES + 1];
  const int n_rings = min(a.ring_off[a.n], a.max_rings);
  for (int i = blockIdx.x; i < n_rings; i += gridDim.x) {
    int lo = 0, hi = a.n;  // frame f: ring_off[f] <= i < ring_off[f + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (a.ring_off[mid] <= i) lo = mid; else hi = mid;
    }
    const int f = lo;
    const double cx = a.rings[i].cx, cy = a.rings[i].cy, rho = a.rings[i].r;
    const double ds = a.dscore ? (double)a.dscore[i] : 1.0;
    const double sig = a.sig_a * rho + a.sig_b;
    const double den = 2.0 * sig * sig;
    // Votes farther than cut from the centre are left out: each of their
    // Gaussian factors is below e^-40.5 < 3e-18 (corners lie within sqrt 2
    // of the vote), so all of them together change a score by < 1e-12 of
    // its value for any frame the records fit.
    const double cut = 9.0 * sig + 1.5;
    const int cnt = min(a.count[f], a.cap);
    const size_t base = (size_t)f * a.cap;
    // A vote lies rho from its pixel, so only the tiles within rho + cut of
    // the centre can contribute; their record ranges, flattened.
    const double reach = rho + cut + 2.0;
    const double ftx0 = floor((cx - reach) / SOFT_T), ftx1 = floor((cx + reach) / SOFT_T);
    const double fty0 = floor((cy - reach) / SOFT_T), fty1 = floor((cy + reach) / SOFT_T);
    const int tx0 = (int)fmax(ftx0, 0.0), tx1 = (int)fmin(ftx1, (double)(a.n_tx - 1));
    const int ty0 = (int)fmax(fty0, 0.0), ty1 = (int)fmin(fty1, (double)(a.n_ty - 1));
    const bool finite = isfinite(cx) && isfinite(cy) && isfinite(reach);
    const int ntx = tx1 - tx0 + 1, nty = ty1 - ty0 + 1;
    const bool tiled = finite && ntx > 0 && nty > 0 && ntx * nty <= SOFT_MAX_TILES;
    int total = cnt;  // not tiled: every record of the frame
    if (finite && (ntx <= 0 || nty <= 0)) total = 0;
    if (tiled) {
      const int nt = ntx * nty;
      for (int t = threadIdx.x; t < nt; t += blockDim.x) {
        const size_t ti = ((size_t)f * a.n_ty + ty0 + t / ntx) * a.n_tx + tx0 + t % ntx;
        s_off[t] = a.tile_off[ti];
        s_pre[t + 1] = a.tile_cnt[ti];
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        s_pre[0] = 0;
        for (int t = 0; t < nt; ++t) s_pre[t + 1] += s_pre[t];
      }
      __syncthreads();
      total = s_pre[nt];
    }
    const double sa = a.sig_ann, sa2 = sa * sa;
    double T = 0.0, Tcx = 0.0, Tcy = 0.0, Tsig = 0.0, Trho = 0.0;
    double TAcx = 0.0, TAcy = 0.0, TArho = 0.0;  // through the annulus weights' dependence on (c, rho)
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
      int j = q;
      if (tiled) {  // the tile t with s_pre[t] <= q < s_pre[t + 1]
        int lo = 0, hi = ntx * nty;
        while (hi - lo > 1) {
          const int mid = (lo + hi) >> 1;
          if (s_pre[mid] <= q) lo = mid; else hi = mid;
        }
        j = s_off[lo] + (q - s_pre[lo]);
      }
      const size_t g = base + j;
      const uint32_t xy = a.xy[g];
      const double px = (double)(xy & 0xffffu), py = (double)(xy >> 16);
      const double X = a.rX[g], Y = a.rY[g], m = a.rm[g];
      // the pixel's annulus weight; a pixel farther than 9 sa from the
      // circle is left out (its weight is below e^-40.5 < 3e-18)
      const double ddx = px - cx, ddy = py - cy;
      const double dist = sqrt(ddx * ddx + ddy * ddy);
      const double e = dist - rho;
      if (!(fabs(e) <= 9.0 * sa)) continue;
      const double A = score_exp(-(e * e) / (2.0 * sa2));
      double tp = 0.0, tcx = 0.0, tcy = 0.0, tsig = 0.0, trho = 0.0;
      double gk = 0.0, gX = 0.0, gY = 0.0;
      for (int s = -1; s <= 1; s += 2) {
        const double vx = px + s * rho * X, vy = py + s * rho * Y;
        const double ex = vx - cx, ey = vy - cy;
        if (ex * ex + ey * ey > cut * cut) continue;
        const double x0 = floor(vx), y0 = floor(vy);
        const double fx = vx - x0, fy = vy - y0;
        for (int oy = 0; oy < 2; ++oy)
          for (int ox = 0; ox < 2; ++ox) {
            const double qx = x0 + ox, qy = y0 + oy;
            if (qx < 0.0 || qx > (double)(a.W - 1) || qy < 0.0 || qy > (double)(a.H - 1)) continue;
            const double wx = ox ? fx : 1.0 - fx, wy = oy ? fy : 1.0 - fy;
            const double dxq = qx - cx, dyq = qy - cy;
            const double d2 = dxq * dxq + dyq * dyq;
            const double G = score_exp(-d2 / den);
            const double mwG = m * wx * wy * G;
            tp += mwG;
            tcx += mwG * dxq;          // x 1/sig^2 below
            tcy += mwG * dyq;
            tsig += mwG * d2;          // x 1/sig^3 below
            // d w / d v: the cell corner is fixed, w = wx wy
            const double dwdvx = (ox ? 1.0 : -1.0) * wy, dwdvy = wx * (oy ? 1.0 : -1.0);
            const double mG = m * G;
            trho += mG * (dwdvx * s * X + dwdvy * s * Y);
            if (a.accumulate) {
              gk += wx * wy * G;
              gX += mG * dwdvx * s * rho;
              gY += mG * dwdvy * s * rho;
            }
          }
      }
      T += A * tp;
      Tcx += A * tcx;
      Tcy += A * tcy;
      Tsig += A * tsig;
      Trho += A * trho;
      // dA/dc = A (-e / sa^2) (c - p) / |p - c|, dA/drho = A e / sa^2
      if (dist > 0.0) {
        const double fa = A * (-e / sa2) / dist;
        TAcx += tp * fa * (cx - px);
        TAcy += tp * fa * (cy - py);
      }
      TArho += tp * A * e / sa2;
      if (a.accumulate && (gk != 0.0 || gX != 0.0 || gY != 0.0)) {
        const double dm = -m * (1.0 - m) / a.temp;  // dm/dk
        atomicAdd(&a.gk[g], ds * A * gk * dm / rho);
        atomicAdd(&a.gX[g], ds * A * gX / rho);
        atomicAdd(&a.gY[g], ds * A * gY / rho);
      }
    }
    T = block_sum(T, red);
    Tcx = block_sum(Tcx, red);
    Tcy = block_sum(Tcy, red);
    Tsig = block_sum(Tsig, red);
    Trho = block_sum(Trho, red);
    TAcx = block_sum(TAcx, red);
    TAcy = block_sum(TAcy, red);
    TArho = block_sum(TArho, red);
    if (threadIdx.x == 0) {
      const double s2 = sig * sig;
      const double score = T / rho;
      // dScore/drho: through the vote positions, sigma(rho), the annulus and the 1/rho
      const double dT_drho = Trho + Tsig / (s2 * sig) * a.sig_a + TArho;
      if (a.score) a.score[i] = (float)score;
      if (a.dparams) {
        a.dparams[3 * i + 0] = (float)(ds * (Tcx / s2 + TAcx) / rho);
        a.dparams[3 * i + 1] = (float)(ds * (Tcy / s2 + TAcy) / rho);
        a.dparams[3 * i + 2] = (float)(ds * (dT_drho / rho - T / (rho * rho)));
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_soft_score(const SoftArgs& a, const int* counts, int* ring_off, cudaStream_t st) {
  k_soft_offsets<<<1, 1024, 0, st>>>(counts, a.n, ring_off);
  k_soft_score<<<152 * 8, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---- S6: chain through the eigen step (per ridge record) -----------------------
// k = (a + c)/2 - R, R = sqrt(((a - c)/2)^2 + b^2); X = sign * v / |v| with
// v = (b, k - a) or (k - c, b); d(v/|v|) = (I - u u^T) dv / |v|.
__global__ void k_soft_chain(SoftArgs a) {
  const size_t plane = (size_t)a.H * a.W;
  const size_t total = (size_t)a.n * a.cap;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(g / a.cap), j = (int)(g - (size_t)f * a.cap);
    if (j >= min(a.count[f], a.cap)) continue;
    const double A = a.ra[g], B = a.rb[g], C = a.rc[g], k = a.rk[g];
    const double hd = 0.5 * (A - C);
    const double R = sqrt(hd * hd + B * B);
    const double dka = 0.5 - 0.5 * hd / R, dkc = 0.5 + 0.5 * hd / R, dkb = -B / R;
    const bool use1 = a.flags[g] & 1;
    const double sgn = (a.flags[g] & 2) ? -1.0 : 1.0;
    const double vx = use1 ? B : k - C, vy = use1 ? k - A : B;
    const double nv = sqrt(vx * vx + vy * vy);
    const double ux = vx / nv, uy = vy / nv;
    // gradient with respect to v: (I - u u^T) (sgn g_X) / |v|
    const double hx = sgn * a.gX[g], hy = sgn * a.gY[g];
    const double dot = ux * hx + uy * hy;
    const double gvx = (hx - ux * dot) / nv, gvy = (hy - uy * dot) / nv;
    // dv/d(a, b, c)
    double ga, gb, gc;
    if (use1) {  // v = (b, k - a)
      ga = gvy * (dka - 1.0);
      gb = gvx + gvy * dkb;
      gc = gvy * dkc;
    } else {     // v = (k - c, b)
      ga = gvx * dka;
      gb = gvx * dkb + gvy;
      gc = gvx * (dkc - 1.0);
    }
    const double gk = a.gk[g];
    ga += gk * dka;
    gb += gk * dkb;
    gc += gk * dkc;
    const uint32_t xy = a.xy[g];
    const size_t p = (size_t)f * plane + (size_t)(xy >> 16) * a.W + (xy & 0xffffu);
    a.a[p] = ga;  // the Hessian images now hold d/d(Lxx, Lxy, Lyy)
    a.b[p] = gb;
    a.c[p] = gc;
  }
}

// ---- S7: adjoint of the reflect-101 correlations -------------------------------
// Forward along one axis: out[i] = sum_t k[t] in[refl(i + t)], |t| <= r.
// Adjoint at j: the outputs i whose tap t reads j directly (i + t = j), by
// the reflection below 0 (i + t = -j, j > 0) or above N - 1
// (i + t = 2 (N - 1) - j, j < N - 1).
__device__ __forceinline__ double adj1d(const double* src, size_t stride, int N, int j, const double* k, int r) {
  double s = 0.0;
  for (int t = -r; t <= r; ++t) {
    int i = j - t;
    if (i >= 0 && i < N) s += k[t + r] * src[i * stride];
    if (j > 0) {
      i = -j - t;
      if (i >= 0 && i < N) s += k[t + r] * src[i * stride];
    }
    if (j < N - 1) {
      i = 2 * (N - 1) - j - t;
      if (i >= 0 && i < N) s += k[t + r] * src[i * stride];
    }
  }
  return s;
}

// vertical Sobel adjoints: t0 = s5_y^T dLxx, t1 = d2_y^T dLyy, k = d1_y^T dLxy
__global__ void k_soft_adj_sobel_v(SoftArgs a) {
  const size_t plane = (size_t)a.H * a.W, total = plane * a.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t f = i / plane;
    const size_t r = i - f * plane;
    const int y = (int)(r / a.W), x = (int)(r - (size_t)y * a.W);
    const size_t o = f * plane + x;
    a.t0[i] = adj1d(a.a + o, a.W, a.H, y, c_s5, 2);
    a.t1[i] = adj1d(a.c + o, a.W, a.H, y, c_d2, 2);
    a.k[i] = adj1d(a.b + o, a.W, a.H, y, c_d1, 2);
  }
}

// horizontal Sobel adjoints: dL = (d2_x^T t0 + s5_x^T t1 + d1_x^T k) / 64 -> X
__global__ void k_soft_adj_sobel_h(SoftArgs a) {
  const size_t plane = (size_t)a.H * a.W, total = plane * a.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t row = i / a.W;
    const int x = (int)(i - row * a.W);
    const size_t o = row * a.W;
    a.X[i] = (adj1d(a.t0 + o, 1, a.W, x, c_d2, 2) + adj1d(a.t1 + o, 1, a.W, x, c_s5, 2) +
              adj1d(a.k + o, 1, a.W, x, c_d1, 2)) / 64.0;
  }
}

// Gaussian adjoints: Y = g_y^T X, then dimage = g_x^T Y
__global__ void k_soft_adj_gauss_v(SoftArgs a) {
  const size_t plane = (size_t)a.H * a.W, total = plane * a.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t f = i / plane;
    const size_t r = i - f * plane;
    const int y = (int)(r / a.W), x = (int)(r - (size_t)y * a.W);
    a.Y[i] = adj1d(a.X + f * plane + x, a.W, a.H, y, a.g, a.R);
  }
}

__global__ void k_soft_adj_gauss_h(SoftArgs a) {
  const size_t plane = (size_t)a.H * a.W, total = plane * a.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t row = i / a.W;
    const int x = (int)(i - row * a.W);
    a.dimage[i] = (float)adj1d(a.Y + row * a.W, 1, a.W, x, a.g, a.R);
  }
}

cudaError_t launch_soft_backward_image(const SoftArgs& a, cudaStream_t st) {
  const size_t bytes = sizeof(double) * a.n * (size_t)a.H * a.W;
  cudaError_t e = cudaMemsetAsync(a.a, 0, bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.b, 0, bytes, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.c, 0, bytes, st);
  if (e != cudaSuccess) return e;
  const unsigned grid = 152 * 8;
  k_soft_chain<<<grid, 256, 0, st>>>(a);
  k_soft_adj_sobel_v<<<grid, 256, 0, st>>>(a);
  k_soft_adj_sobel_h<<<grid, 256, 0, st>>>(a);
  k_soft_adj_gauss_v<<<grid, 256, 0, st>>>(a);
  k_soft_adj_gauss_h<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---- refinement: one gradient-ascent step per ring ------------------------------
// The ascent is on the unnormalised vote mass rho * Score: the 1/rho of the
// score compares rings of different radii, but for one ring it pulls the
// maximum in rho inward by about sigma^2 / rho.  Its gradient is
// (rho dS/dc, rho dS/drho + S); with the Newton-like scaling by the
// curvature -rho S / se^2, 1 / se^2 = 1 / sigma(rho)^2 + 1 / sa^2 (the vote
// Gaussian and the annulus both narrow the maximum), the step is
//   delta = step * se^2 / S * (dS/dcx, dS/dcy, dS/drho + S / rho),
// each component at most 0.5 px.
__global__ void k_soft_refine_step(SoftArgs a) {
  const int n_rings = min(a.ring_off[a.n], a.max_rings);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_rings; i += gridDim.x * blockDim.x) {
    rd_ring& q = a.rings_mut[i];
    const float sc = a.score[i];
    if (!(sc > 0.0f)) continue;
    const float sig = a.sig_a * q.r + a.sig_b;
    const float sa = (float)a.sig_ann;
    const float se2 = sig * sig * sa * sa / (sig * sig + sa * sa);
    const float scale = a.step * se2 / sc;
    const float d0 = fminf(fmaxf(scale * a.dparams[3 * i + 0], -0.5f), 0.5f);
    const float d1 = fminf(fmaxf(scale * a.dparams[3 * i + 1], -0.5f), 0.5f);
    const float d2 = fminf(fmaxf(scale * (a.dparams[3 * i + 2] + sc / q.r), -0.5f), 0.5f);
    q.cx += d0;
    q.cy += d1;
    q.r = fmaxf(q.r + d2, 1.0f);
  }
}

cudaError_t launch_soft_refine_step(const SoftArgs& a, cudaStream_t st) {
  k_soft_refine_step<<<152, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rd
