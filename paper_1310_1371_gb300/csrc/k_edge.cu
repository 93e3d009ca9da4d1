// k_edge.cu -- directed-edge feature stage (the variant of the Additional
// notes: the gradient replaces the Hessian, and the gradient magnitude,
// replacing k-, must be a local maximum along the gradient direction).
//
// Same numerical contract as the ridge stage: the Gaussian smoothing of an
// integer frame is exact (u32 then u64), the first-order 5x5 Sobel of L' is an
// exact int64, and (Gx, Gy) = (Gx', Gy') / (128 S^2), |grad|, the unit
// direction and every decision are then taken in double precision with one
// correctly rounded operation per step, in the order of the definition, so
// the edge set is the definition's.  The records go into the ridge-record
// lists that binning, voting and fitting read; each also keeps its exact
// double direction, which the voting stage's double-precision path uses.
#include "rd_internal.cuh"

namespace rd {

__device__ __forceinline__ int erefl(int i, int n) {
  i = i < 0 ? -i : i;
  return i >= n ? 2 * (n - 1) - i : i;
}

template <typename T>
__global__ void k_edge_h(EdgeArgs a) {
  const size_t total = (size_t)a.n * a.H * a.W;
  const T* img = reinterpret_cast<const T*>(a.frames);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t row = i / a.W;
    const int x = (int)(i - row * a.W);
    const T* r = img + row * a.W;
    uint32_t s = 0;
    for (int t = -a.taps.R; t <= a.taps.R; ++t) s += (uint32_t)a.taps.q[t + a.taps.R] * (uint32_t)r[erefl(x + t, a.W)];
    a.hp[i] = s;
  }
}

__global__ void k_edge_v(EdgeArgs a) {
  const size_t plane = (size_t)a.H * a.W, total = plane * a.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t f = i / plane;
    const size_t r = i - f * plane;
    const int y = (int)(r / a.W), x = (int)(r - (size_t)y * a.W);
    const uint32_t* col = a.hp + f * plane + x;
    unsigned long long s = 0;
    for (int t = -a.taps.R; t <= a.taps.R; ++t)
      s += (unsigned long long)(uint32_t)a.taps.q[t + a.taps.R] * col[(size_t)erefl(y + t, a.H) * a.W];
    a.L[i] = s;
  }
}

__global__ void k_edge_grad(EdgeArgs a) {
  const long long s5[5] = {1, 4, 6, 4, 1}, d1[5] = {-1, -2, 0, 2, 1};
  const size_t plane = (size_t)a.H * a.W, total = plane * a.n;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t f = i / plane;
    const size_t r = i - f * plane;
    const int y = (int)(r / a.W), x = (int)(r - (size_t)y * a.W);
    const unsigned long long* L = a.L + f * plane;
    long long gx = 0, gy = 0;
    for (int dy = 0; dy < 5; ++dy) {
      const unsigned long long* row = L + (size_t)erefl(y + dy - 2, a.H) * a.W;
      long long sx = 0, dx1 = 0;
      for (int dx = 0; dx < 5; ++dx) {
        const long long l = (long long)row[erefl(x + dx - 2, a.W)];
        sx += s5[dx] * l;
        dx1 += d1[dx] * l;
      }
      gx += s5[dy] * dx1;
      gy += d1[dy] * sx;
    }
    const double Gx = d_div(__ll2double_rn(gx), a.D64), Gy = d_div(__ll2double_rn(gy), a.D64);
    const double g = d_sqrt(d_add(d_mul(Gx, Gx), d_mul(Gy, Gy)));
    // the direction is needed only where the pixel can be an edge (|grad|
    // above the threshold); the magnitude everywhere (bilinear samples)
    double X = 0.0, Y = 0.0;
    if (g != 0.0 && g > a.thresh) {
      X = d_div(Gx, g);
      Y = d_div(Gy, g);
      if (X < 0.0 || (X == 0.0 && Y < 0.0)) {
        X = -X;
        Y = -Y;
      }
    }
    a.g[i] = g;
    a.X[i] = X;
    a.Y[i] = Y;
  }
}

// One CTA per 32 x 32 stencil tile: the edge test of its pixels, then the
// records in row-major order inside the tile (as the ridge stage).
__global__ void __launch_bounds__(256) k_edge_mask(EdgeArgs a) {
  __shared__ int sScan[ST_THREADS / 32 + 1];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int f = blockIdx.z, x0 = blockIdx.x * ST_TW, y0 = blockIdx.y * ST_TH;
  const size_t plane = (size_t)a.H * a.W;
  const double* G = a.g + f * plane;
  bool flag[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int pi = tid + j * ST_THREADS;
    const int tx = pi % ST_TW, ty = pi / ST_TW;
    const int x = x0 + tx, y = y0 + ty;
    bool e = false;
    if (x < a.W && y < a.H) {
      const size_t i = (size_t)y * a.W + x;
      const double gp = G[i], X = a.X[f * plane + i], Y = a.Y[f * plane + i];
      if (gp > a.thresh && !(X == 0.0 && Y == 0.0)) {
        e = true;
        for (int s = 0; s < 2 && e; ++s) {
          const double qx = s == 0 ? d_add((double)x, X) : d_sub((double)x, X);
          const double qy = s == 0 ? d_add((double)y, Y) : d_sub((double)y, Y);
          if (qx < 0.0 || qx > (double)(a.W - 1) || qy < 0.0 || qy > (double)(a.H - 1)) {
            e = false;
            break;
          }
          const double xf = floor(qx), yf = floor(qy);
          const double fx = d_sub(qx, xf), fy = d_sub(qy, yf);
          const int xa = (int)xf, ya = (int)yf;
          const int xb = min(xa + 1, a.W - 1), yb = min(ya + 1, a.H - 1);
          const double gt = bilinear64(fx, fy, G[(size_t)ya * a.W + xa], G[(size_t)ya * a.W + xb],
                                       G[(size_t)yb * a.W + xa], G[(size_t)yb * a.W + xb]);
          e = s == 0 ? (gp > gt) : (gp >= gt);
        }
      }
    }
    flag[j] = e;
  }
  int pos[4], base = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const unsigned bal = __ballot_sync(0xffffffffu, flag[j]);
    if (lane == 0) sScan[warp] = __popc(bal);
    __syncthreads();
    int wpre = 0, tot = 0;
    for (int w = 0; w < ST_THREADS / 32; ++w) {
      const int c = sScan[w];
      wpre += (w < warp) ? c : 0;
      tot += c;
    }
    pos[j] = base + wpre + __popc(bal & ((1u << lane) - 1u));
    base += tot;
    __syncthreads();
  }
  const int total = base;
  const int tile = blockIdx.y * a.rl.n_stx + blockIdx.x;
  const size_t tbase = (size_t)f * a.rl.n_stx * a.rl.n_sty + tile;
  if (tid == 0) {
    const int start = total ? atomicAdd(&a.rl.count[f], total) : 0;
    sScan[ST_THREADS / 32] = start;
    const int keep = max(0, min(total, a.rl.cap - start));
    if (keep < total) atomicOr(&a.stats->overflow, 1);
    a.rl.tile_off[tbase] = total ? start : 0;
    a.rl.tile_cnt[tbase] = keep;
    if (total) atomicAdd(&a.stats->ridge, (unsigned long long)total);
  }
  __syncthreads();
  const int start = sScan[ST_THREADS / 32];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!flag[j]) continue;
    const int o = start + pos[j];
    if (o >= a.rl.cap) continue;
    const int pi = tid + j * ST_THREADS;
    const int x = x0 + pi % ST_TW, y = y0 + pi / ST_TW;
    const size_t i = f * plane + (size_t)y * a.W + x;
    const size_t g = (size_t)f * a.rl.cap + o;
    const double X = a.X[i], Y = a.Y[i];
    // the double direction as a float pair: |X - (hi + lo)| <= 2^-49
    const float xh = __double2float_rn(X), yh = __double2float_rn(Y);
    const float xl = __double2float_rn(X - (double)xh), yl = __double2float_rn(Y - (double)yh);
    const float eXr = 7.105427e-15f;  // 2^-47
    const float kfast = 1.25f * (fmaxf(fabsf(xl), fabsf(yl)) + eXr + 5.9604645e-8f) + 5.9604645e-8f;
    const float kref = 1.25f * eXr + 2.842171e-14f;
    a.rl.xy[g] = (uint32_t)x | ((uint32_t)y << 16);
    a.rl.dir[g] = make_float4(xh, yh, xl, yl);
    a.rl.kvote[g] = make_float2(kfast, kref);
    a.rl.hess[3 * g + 0] = 0;
    a.rl.hess[3 * g + 1] = 0;
    a.rl.hess[3 * g + 2] = 0;
    a.rl.x64[g] = make_double2(X, Y);
  }
}

cudaError_t launch_edge(const EdgeArgs& a, int dtype, cudaStream_t st) {
  const unsigned grid = 152 * 8;
  if (dtype == RD_U8)
    k_edge_h<uint8_t><<<grid, 256, 0, st>>>(a);
  else
    k_edge_h<uint16_t><<<grid, 256, 0, st>>>(a);
  k_edge_v<<<grid, 256, 0, st>>>(a);
  k_edge_grad<<<grid, 256, 0, st>>>(a);
  const dim3 tiles(a.rl.n_stx, a.rl.n_sty, a.n);
  k_edge_mask<<<tiles, ST_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rd
