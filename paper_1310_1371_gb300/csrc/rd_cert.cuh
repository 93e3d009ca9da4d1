// rd_cert.cuh -- certified FP32 decisions of the directed-ridge test and
// their exact double-precision fallback, shared by the detector's stencil
// stage (integer frames) and the soft score's (float frames).
//
// Method: Results ("Directed ridge detection & votes collection": k- < tau
// and a local minimum of k- along X-); Detailed algorithm step 2.  Each FP32
// quantity comes with a rigorous bound on its distance to the value the
// double-precision definition computes; a decision whose margin does not
// clear its bound is reported as undecided and re-taken in FP64.
#pragma once
#include "rd_internal.cuh"

namespace rd {

constexpr float U32 = 5.9604645e-8f;  // 2^-24

// FP32 k- of (a, b, c) with ek bounding its FP32 evaluation error plus the
// definition's own double rounding, 16 u (|a| + |b| + |c|); the caller adds
// the effect of the inputs' error (3 delta, see hess32).
__device__ __forceinline__ void eig32_k(float a, float b, float c, float& k, float& ek, float& hdf, float& rad) {
  float htr = (a + c) * 0.5f;
  hdf = (a - c) * 0.5f;
  rad = sqrtf(hdf * hdf + b * b);
  k = htr - rad;
  float M = fabsf(a) + fabsf(b) + fabsf(c);
  ek = M * (16.0f * U32) + 1e-30f;
}

// Stable FP32 X- (no cancellation: the large component is |hdf| + rad) with a
// bound eX on each component's distance to the exact direction (same sign).
// delta bounds the inputs' absolute error (see hess32): v = (b, -w) or
// (-w, b), w = |hdf| + rad, moves by at most sqrt(1 + (1 + sqrt 2)^2) delta
// < 2.62 delta, and v / |v| by twice that over |v|.  Returns false where
// |v| is too small for a bound (the exactly degenerate case among them).
__device__ __forceinline__ bool eig32_dir(float b, float hdf, float rad, float M, float delta, float& X, float& Y,
                                          float& eX) {
  float w = fabsf(hdf) + rad;
  float vx, vy;
  if (hdf >= 0.0f) {
    vx = b;
    vy = -w;
  } else {
    vx = -w;
    vy = b;
  }
  float nrm = sqrtf(vx * vx + vy * vy);
  if (!(nrm > 4.0f * delta) || !(nrm > 0.0f)) return false;
  X = vx / nrm;
  Y = vy / nrm;
  if (X < 0.0f || (X == 0.0f && Y < 0.0f)) {
    X = -X;
    Y = -Y;
  }
  eX = (M * (16.0f * U32)) / nrm + 4.0f * U32 + 6.0f * delta / (nrm - 3.0f * delta);
  return true;
}

// Exact (double-precision definition) ridge test of the pixel (gx, gy) from
// the exact k- of its 3x3 neighbourhood kn (row-major, centre kn[4]) and its
// exact X- = (X, Y): k- < tau, then the bilinear samples at p + X- (strict)
// and p - X- (non-strict); a sample outside the image makes it no ridge.
static __device__ __noinline__ bool ridge_exact_nb(const double* kn, double X, double Y, bool degenerate, int gx, int gy,
                                            int H, int W, double tau) {
  const double k = kn[4];
  if (!(k < tau) || degenerate) return false;
  for (int s = 0; s < 2; ++s) {
    double qx = s == 0 ? d_add((double)gx, X) : d_sub((double)gx, X);
    double qy = s == 0 ? d_add((double)gy, Y) : d_sub((double)gy, Y);
    if (qx < 0.0 || qx > (double)(W - 1) || qy < 0.0 || qy > (double)(H - 1)) return false;
    double x0f = floor(qx), y0f = floor(qy);
    double fx = d_sub(qx, x0f), fy = d_sub(qy, y0f);
    int cx0 = (int)x0f, cy0 = (int)y0f;
    int cx1 = min(cx0 + 1, W - 1), cy1 = min(cy0 + 1, H - 1);
    if (fx == 0.0) cx1 = cx0;  // zero-weight corner: any finite value gives the same sum
    if (fy == 0.0) cy1 = cy0;
    // |X|, |Y| <= 1, so every corner is within one pixel of (gx, gy)
    const int i0 = (cy0 - gy + 1) * 3, i1 = (cy1 - gy + 1) * 3, j0 = cx0 - gx + 1, j1 = cx1 - gx + 1;
    double kt = bilinear64(fx, fy, kn[i0 + j0], kn[i0 + j1], kn[i1 + j0], kn[i1 + j1]);
    if (s == 0 ? !(k < kt) : !(k <= kt)) return false;
  }
  return true;
}

// 0 = certainly not a ridge, 1 = certainly a ridge, 2 = undecided in FP32.
// Each sample p +/- X- is interpolated on the cell that holds the FP32
// sample.  The exact sample lies in the box of half-width eX around it and
// within one pixel of p (|X-| <= 1 component-wise).  Where the box crosses a
// cell edge (the FP32 sample is within eX of an integer, a test exact by
// Sterbenz), the corner set grows along that axis to all three columns (or
// rows) within one pixel of p, clipped to the image.  The bilinear
// interpolant is continuous, and along an axis-parallel path its slope never
// exceeds the spread (max - min) of the corners of the cells it crosses, so
// between the two samples it moves by at most 2 eX times the spread of the
// corner set; the corner errors and the interpolation's rounding are bounded
// over the same set.  On the image's border rows and columns a box that
// reaches the border stays undecided (the exact sample may lie outside).
__device__ __forceinline__ int ridge_fast(const float* sK, const float* sE, int stride, int hy, int hx, int gx, int gy,
                                          int H, int W, float k, float ek, float tau, float X, float Y, float eX) {
  int verdict = 1;
  for (int s = 0; s < 2; ++s) {
    float ox = s == 0 ? X : -X, oy = s == 0 ? Y : -Y;
    float lowx = (float)(-gx), highx = (float)(W - 1 - gx);
    float lowy = (float)(-gy), highy = (float)(H - 1 - gy);
    if (ox < lowx - eX || ox > highx + eX || oy < lowy - eX || oy > highy + eX) return 0;
    // Off the border rows and columns the exact sample is inside the image
    // (|X-| <= 1 component-wise), so only there can a box near a border hide
    // a sample outside it.
    const bool bx = gx == 0 || gx == W - 1, by = gy == 0 || gy == H - 1;
    if (eX > 0.0f && ((bx && (ox <= lowx + eX || ox >= highx - eX)) || (by && (oy <= lowy + eX || oy >= highy - eX))))
      return 2;
    float flx = floorf(ox), fly = floorf(oy);
    float fx = ox - flx, fy = oy - fly;
    int cx0 = gx + (int)flx, cy0 = gy + (int)fly;
    int cx1 = fx == 0.0f ? cx0 : min(cx0 + 1, W - 1);
    int cy1 = fy == 0.0f ? cy0 : min(cy0 + 1, H - 1);
    int lx0 = hx + (cx0 - gx), lx1 = hx + (cx1 - gx), ly0 = hy + (cy0 - gy), ly1 = hy + (cy1 - gy);
    int i00 = ly0 * stride + lx0, i01 = ly0 * stride + lx1, i10 = ly1 * stride + lx0, i11 = ly1 * stride + lx1;
    float k00 = sK[i00], k01 = sK[i01], k10 = sK[i10], k11 = sK[i11];
    float gxw = 1.0f - fx, gyw = 1.0f - fy;
    float kt = gyw * (gxw * k00 + fx * k01) + fy * (gxw * k10 + fx * k11);
    float kmax = fmaxf(fmaxf(k00, k01), fmaxf(k10, k11));
    float kmin = fminf(fminf(k00, k01), fminf(k10, k11));
    float ekc = fmaxf(fmaxf(sE[i00], sE[i01]), fmaxf(sE[i10], sE[i11]));
    // the corner set grows where the box crosses a cell edge (rare): all
    // columns (rows) within one pixel of p along that axis, in the image
    const bool ex = eX > 0.0f && fabsf(ox - rintf(ox)) <= eX;
    const bool ey = eX > 0.0f && fabsf(oy - rintf(oy)) <= eX;
    if (ex || ey) {
      const int xa = ex ? max(-1, -gx) : cx0 - gx, xb = ex ? min(1, W - 1 - gx) : cx1 - gx;
      const int ya = ey ? max(-1, -gy) : cy0 - gy, yb = ey ? min(1, H - 1 - gy) : cy1 - gy;
      for (int dy = ya; dy <= yb; ++dy) {
        const int row = (hy + dy) * stride + hx;
        for (int dx = xa; dx <= xb; ++dx) {
          const float kc = sK[row + dx];
          kmax = fmaxf(kmax, kc);
          kmin = fminf(kmin, kc);
          ekc = fmaxf(ekc, sE[row + dx]);
        }
      }
    }
    float kabs = fmaxf(fabsf(kmax), fabsf(kmin));
    float m = ek + ekc + 2.0f * eX * (kmax - kmin) + 8.0f * U32 * kabs + 1e-30f;
    float diff = kt - k;  // need k < kt (s = +) or k <= kt (s = -)
    if (diff < -m) return 0;
    if (!(diff > m)) verdict = 2;
  }
  return verdict;
}

// FP32 row filters of one Hessian-tile row point from five consecutive
// rounded L values: s = l0 + 4 (l1 + l3) + 6 l2 + l4, d2 = l0 - 2 l2 + l4,
// d1 = (l4 - l0) + 2 (l3 - l1), each operation correctly rounded in the
// written order.
__device__ __forceinline__ void row_filters32(const float* row, float& rs, float& rd2, float& rd1) {
  const float l0 = row[0], l1 = row[1], l2 = row[2], l3 = row[3], l4 = row[4];
  const float e = __fadd_rn(l0, l4);
  rs = __fmaf_rn(6.0f, l2, __fmaf_rn(4.0f, __fadd_rn(l1, l3), e));
  rd2 = __fmaf_rn(-2.0f, l2, e);
  rd1 = __fmaf_rn(2.0f, __fsub_rn(l3, l1), __fsub_rn(l4, l0));
}

// FP32 Hessian entries (a, b, c) = fl(H) x fl(1/D) from the row filters of
// five consecutive rows: the column filters s over d2 (Lxx), d2 over s (Lyy)
// and d1 over d1 (Lxy), each operation correctly rounded in the written
// order (no contraction).
__device__ __forceinline__ void hess32_v(float x0, float x1, float x2, float x3, float x4, float y0, float y2, float y4,
                                         float z0, float z1, float z3, float z4, float invD, float& fa, float& fb,
                                         float& fc) {
  const float hxx = __fmaf_rn(6.0f, x2, __fmaf_rn(4.0f, __fadd_rn(x1, x3), __fadd_rn(x0, x4)));
  const float hyy = __fmaf_rn(-2.0f, y2, __fadd_rn(y0, y4));
  const float hxy = __fmaf_rn(2.0f, __fsub_rn(z3, z1), __fsub_rn(z4, z0));
  fa = __fmul_rn(hxx, invD);
  fb = __fmul_rn(hxy, invD);
  fc = __fmul_rn(hyy, invD);
}

// The same at Hessian-tile index c0 from row-filter arrays (row stride st),
// over rows c0, c0 + st, ..., c0 + 4 st.
__device__ __forceinline__ void hess32(const float* Rs, const float* Rd2, const float* Rd1, int st, int c0, float invD,
                                       float& fa, float& fb, float& fc) {
  hess32_v(Rd2[c0], Rd2[c0 + st], Rd2[c0 + 2 * st], Rd2[c0 + 3 * st], Rd2[c0 + 4 * st], Rs[c0], Rs[c0 + 2 * st],
           Rs[c0 + 4 * st], Rd1[c0], Rd1[c0 + st], Rd1[c0 + 3 * st], Rd1[c0 + 4 * st], invD, fa, fb, fc);
}

}  // namespace rd
