// rd_internal.cuh -- structures and device helpers shared by the detector's
// kernels.  Nothing here is part of the public ABI (include/rd.h).
//
// Numerical contract.  Integer frames are smoothed with integer Gaussian
// taps, so the Hessian (Hxx', Hyy', Hxy') = 64 S^2 (Lxx, Lyy, Lxy) is an exact
// int64 (Methods: Gaussian convolution, then the 5x5 second-order Sobel),
// formed where a decision or a record needs it.  Every decision (k- < tau,
// the local-minimum test along X-, the rounding of each vote to a bin,
// annulus membership) is taken in fast FP32 arithmetic together with a
// rigorous bound on its error; when the bound does not separate the value
// from the decision boundary the decision is re-taken by an FP64 evaluation
// that performs the same IEEE operations in the same order as the definition
// (helpers named *64 below), so the decision equals that of the
// double-precision definition.  Vote directions carry a double-float
// (hi + lo) refinement so that only a tiny fraction of the votes reach FP64.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <climits>
#include <nvtx3/nvToolsExt.h>

#include "rd.h"

namespace rd {

// Host-side NVTX range over a scope: profilers (ncu --nvtx, nsys) attribute
// the kernels enqueued inside it to the named stage.  Without an attached
// tool the calls return at once.
struct NvtxScope {
  explicit NvtxScope(const char* name) { nvtxRangePushA(name); }
  ~NvtxScope() { nvtxRangePop(); }
  NvtxScope(const NvtxScope&) = delete;
  NvtxScope& operator=(const NvtxScope&) = delete;
};

constexpr int GAUSS_BITS = 19;     // Gaussian taps: integers summing to ~2^19
constexpr int SMOOTH_BITS = 16;    // level-smoothing weights: peak 2^16
constexpr int MAX_RG = 16;         // Gaussian half-width ceil(4 sigma), sigma <= 4
constexpr int ST_TW = 32;          // stencil tile (output pixels)
constexpr int ST_TH = 32;
constexpr int ST_THREADS = 256;
constexpr int ACC_T_LARGE = 128;   // supported accumulator tile edges (the dense fallback
constexpr int ACC_T = 96;          // kernel splits 128-pixel tiles into four 64-pixel ones)
constexpr int ACC_T_MID = 80;
constexpr int ACC_T_SMALL = 64;
constexpr int VOTE_THREADS = 256;
constexpr int MAX_RS = 40;         // level smoothing half-width ceil(3 sigma(r))
constexpr int SLAB_LEVELS = 12;    // peak levels per r-slab of the smaller-tile fallbacks
constexpr int MAX_SLAB_LEVELS = 64;
constexpr int DEFAULT_SLAB_LEVELS = 32;  // the automatic geometry's slab depth
constexpr int FIT_WARPS = 8;
constexpr int BIN_SMEM_MAX = 8192;  // bins per frame up to which binning counts in shared memory
constexpr int BIN_GRID_MAX = 64;    // binning CTAs per frame in that mode
// Vote-rounding margin coefficient shared by every well-conditioned ridge
// pixel: 1.25 (|X_lo| + e_X + 2^-24) + 2^-24 with |X_lo| <= 2^-25 and the
// direction error e_X <= 5e-12 (condition number <= 1e3).  Pixels whose own
// coefficient exceeds it always take the exact path.
constexpr float KF_CONST = 1.72e-7f;

// Debug build (compile with -DRD_CHECK): data-dependent indices into shared
// and global buffers are checked before use.  A failed check sets
// RD_OVF_CHECK in the call's statistics and the access is skipped; nothing
// traps.  In the normal build the checks compile to nothing.
#ifdef RD_CHECK
#define RD_GUARD(cond, stats) ((cond) ? true : (atomicOr(&(stats)->overflow, RD_OVF_CHECK), false))
#else
#define RD_GUARD(cond, stats) true
#endif

struct DevStats {
  unsigned long long ridge, votes, peaks, fallbacks;
  int overflow;
  int pad;
  unsigned long long hotspots, smooth_macs;  // each hotspot counted once (tile interior, owned level)
};

struct GaussTaps {
  int R;                           // half-width
  int32_t q[2 * MAX_RG + 1];
};

// Ridge list of a batch: frame f's records live at [f*cap, f*cap + count[f]).
struct RidgeList {
  uint32_t* xy;      // x | y << 16
  float4* dir;       // (Xhi, Yhi, Xlo, Ylo): unit direction X- as a double-float
  float2* kvote;     // per-record vote-rounding margins (fast FP32, double-float)
  long long* hess;   // exact Hessian (Hxx', Hyy', Hxy'), 3 per record
  int* count;        // per frame (atomic; may exceed cap)
  int* tile_off;     // per frame and stencil tile: first record
  int* tile_cnt;     // per frame and stencil tile: record count
  double2* x64;      // directed-edge records: the exact double direction (null for ridges)
  int cap;
  int n_stx, n_sty;  // stencil tiles per frame
};

// ---------------------------------------------------------------------------
// kernel argument blocks and launchers (one definition for every TU)
// ---------------------------------------------------------------------------
struct StencilArgs {
  const void* frames;
  int n, H, W;
  GaussTaps taps;
  // directed ridges: tau and D = 64 S^2 (Lxx = Hxx' / D).  Directed edges
  // (edge = 1): -(gradient threshold) and D = 128 S^2 ((Gx, Gy) = (Gx', Gy') / D),
  // the stage then testing -|grad| as it tests k-.
  int edge;
  float tau;
  double tau64;
  double D64;
  float invD;     // fl(1 / D)
  RidgeList rl;
  DevStats* stats;
  uint32_t narrow_max;  // largest input value for which the exact Gaussian's pair sums fit u32
                        // (set by launch_stencil from the taps: 2 S narrow_max < 2^32)
  int vec_rows;         // frames and rows start on 16-byte boundaries (set by launch_stencil)
};

struct BinArgs {
  RidgeList rl;
  int n_frames, H, W;          // H, W: the accumulator grid in cells (the image for lc = 0)
  int n_atx, n_aty, n_slabs, T;
  int lc;                      // log2 of the cell edge in px (coarse parameter space); 0, 1 or 2
  float inv_c;                 // 2^-lc
  const int4* slabs;           // (lo, hi, halo, 0): peak levels lo..hi, votes lo-1..hi+1
  int* bin_cnt;
  const int* bin_off;
  int* bin_fill;
  int* cta_cnt;              // per (frame, bin, CTA of the frame's grid row): entries (null: global counters)
  uint4* pool;               // per entry: int16 x | int16 y << 16 in px relative to the tile region
                             // (origin 2^lc (tx T - h, ty T - h)), s X, s Y,
                             // index << 3 | exact axis << 2 | ill << 1 | (s < 0)
  long long pool_cap;
  DevStats* stats;
};

struct VoteArgs {
  RidgeList rl;
  int n_frames, H, W, n_atx, n_aty, n_slabs, T;  // H, W: the accumulator grid in cells
  int lc;                    // log2 of the cell edge in px (coarse parameter space)
  const int4* slabs;
  const int* bin_cnt;
  const int* bin_off;
  const uint4* pool;
  long long pool_cap;
  const int* q_rad;          // per voting level (index r - (r_min - 1)): R_s
  const int* qq_off;         // per (slab, level lo-1 .. hi+1): offset into qq_tab
  const int2* qq_tab;        // (weight, slab-relative smem offset) per window tap, row-major (dy, dx)
  const int* qp_off;         // per (slab, level): offset into qp_tab (multiple of 4)
  int slab_stride;           // entries per slab in qq_off / qp_off: slab levels + 2
  const uint32_t* qp_tab;    // per level: {0, 0, Q(0,0), 0}, then {o1, o2, Q, 0} per orbit of four taps
  int* queue;                // K4 work queue: non-empty bins, largest first
  int* n_queue;              // its length
  int* queue_head;           // next item to take
  int vote_grid;             // SMs; the persistent K4 grid is this times the resident CTAs per SM
  int* fb_list;              // bins handed to the dense kernel (sparse capacities exceeded)
  int* fb_count;
  int fb_cap, fb_grid;
  int route_dense;           // diagnostics: hand every bin to the dense kernel
  const unsigned long long* nthr;  // per voting level: smallest N passing the float threshold
  int r_min, r_max, vote_thresh;
  int4* peaks;               // per frame: (x, y, r, N)
  int peak_cap;
  int* peak_count;
  DevStats* stats;
  double D64;
  int32_t* dbg_acc;          // optional [levels][H][W] capture of frame 0
  uint32_t* dbg_sm;
  int max_rw, max_qn, max_qp;
  int T_dense, max_rw_dense;  // tile edge and window of the dense fallback kernel
};

struct FitArgs {
  RidgeList rl;
  int n_frames, H, W;
  const int4* peaks;
  const int* peak_count;
  int peak_cap;
  const int* offsets;
  rd_ring* rings;
  int ring_cap;
  float w;            // annulus half-width
  int w_int;          // w is an integer: exact integer membership test
  DevStats* stats;
};

// Soft (differentiable) score path: FP64 images and ridge records of a batch
// of frames, allocated on first use (k_soft.cu).
struct SoftArgs {
  const void* frames;
  int dtype;                  // RD_U8, RD_U16 or RD_F32
  int n, H, W;
  int R;                      // Gaussian half-width
  double g[2 * MAX_RG + 1];   // Gaussian taps Q_i / S
  double tau, temp, sig_a, sig_b;
  double sig_ann;             // the soft annulus's standard deviation: half the annulus half-width w
  // dense FP64 images, n * H * W each
  double *t0, *t1, *a, *b, *c, *k, *X, *Y;
  // ridge records, frame f at [f * cap, f * cap + count[f]); those of 32 x 32
  // tile t of frame f at [tile_off, tile_off + tile_cnt) within the frame's
  int cap;
  int* count;
  int n_tx, n_ty;             // tiles per row and column
  int *tile_off, *tile_cnt;   // n * n_ty * n_tx
  uint32_t* xy;               // x | y << 16
  uint8_t* flags;             // bit 0: eigenvector candidate v1; bit 1: sign flipped
  double *rk, *rX, *rY, *ra, *rb, *rc, *rm;
  double *gk, *gX, *gY;       // accumulated d(sum dscore Score)/d(k, X, Y) per record
  // rings
  const rd_ring* rings;
  rd_ring* rings_mut;
  int n_rings;
  const int* ring_off;        // exclusive prefix of the per-frame ring counts, n + 1
  const float* dscore;        // per ring, or null (1)
  float* score;               // per ring, or null
  float* dparams;             // per ring 3, or null
  float* dimage;              // n * H * W, or null
  int accumulate;             // add record gradients (backward)
  int max_rings;              // rings beyond this index are ignored
  float step;                 // refine step
};

cudaError_t launch_soft_stencil(const SoftArgs& a, cudaStream_t st);
cudaError_t launch_soft_score(const SoftArgs& a, const int* counts, int* ring_off, cudaStream_t st);
cudaError_t launch_soft_backward_image(const SoftArgs& a, cudaStream_t st);
cudaError_t launch_soft_refine_step(const SoftArgs& a, cudaStream_t st);

cudaError_t launch_stencil(const StencilArgs& a, int dtype, cudaStream_t st);
cudaError_t launch_refine(const RidgeList& rl, int n_frames, int n_sm, cudaStream_t st);
cudaError_t launch_bins(const BinArgs& a, int n_sm, cudaStream_t st, long long n_bins, int* block_sums,
                        long long* total_dev);
cudaError_t launch_vote(const VoteArgs& a, long long n_bins, cudaStream_t st);
cudaError_t launch_fit(const FitArgs& a, int4* peaks_mut, int* counts, int* offsets, cudaStream_t st);
size_t stencil_smem_bytes(int R);
size_t vote_smem_bytes(int max_rw, int T, int max_qn);
size_t sparse_smem_bytes(int max_rw, int max_qp);

// ---------------------------------------------------------------------------
// FP64 replicas of the definition (one correctly rounded IEEE op per call)
// ---------------------------------------------------------------------------
__device__ __forceinline__ double d_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double d_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double d_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double d_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double d_sqrt(double a) { return __dsqrt_rn(a); }

struct Eig64 {
  double k, X, Y;
  bool degenerate;
};

// The definition's entries a = Hxx'/D, c = Hyy'/D, b = Hxy'/D and
// k = (a + c)/2 - sqrt(((a - c)/2)^2 + b^2), one correctly rounded
// operation per step.
__device__ inline double eigen64_k(long long hxx, long long hyy, long long hxy, double D, double& a, double& c,
                                   double& b) {
  a = d_div(__ll2double_rn(hxx), D);
  c = d_div(__ll2double_rn(hyy), D);
  b = d_div(__ll2double_rn(hxy), D);
  double half_tr = d_mul(d_add(a, c), 0.5);
  double half_df = d_mul(d_sub(a, c), 0.5);
  double rad = d_sqrt(d_add(d_mul(half_df, half_df), d_mul(b, b)));
  return d_sub(half_tr, rad);
}

// X- from the entries and k: candidates v1 = (b, k - a), v2 = (k - c, b),
// the larger squared norm wins (v1 on a tie); normalised; sign X > 0 or
// (X == 0 and Y > 0).  Degenerate (both candidates zero): never a ridge.
__device__ inline void eigen64_dir(double a, double c, double b, double k, Eig64& e) {
  double v1x = b, v1y = d_sub(k, a);
  double v2x = d_sub(k, c), v2y = b;
  double n1 = d_add(d_mul(v1x, v1x), d_mul(v1y, v1y));
  double n2 = d_add(d_mul(v2x, v2x), d_mul(v2y, v2y));
  bool use1 = n1 >= n2;
  double vx = use1 ? v1x : v2x, vy = use1 ? v1y : v2y, n = use1 ? n1 : n2;
  e.k = k;
  e.degenerate = (n == 0.0);
  if (e.degenerate) {
    e.X = 0.0;
    e.Y = 0.0;
    return;
  }
  double nrm = d_sqrt(n);
  double X = d_div(vx, nrm), Y = d_div(vy, nrm);
  if (X < 0.0 || (X == 0.0 && Y < 0.0)) {
    X = -X;
    Y = -Y;
  }
  e.X = X;
  e.Y = Y;
}

// k- and X- of H = [[a, b], [b, c]] (the two steps above).
__device__ inline Eig64 eigen64(long long hxx, long long hyy, long long hxy, double D) {
  double a, c, b;
  const double k = eigen64_k(hxx, hyy, hxy, D, a, c, b);
  Eig64 e;
  eigen64_dir(a, c, b, k, e);
  return e;
}

// Bilinear sample (1-fy)((1-fx) k00 + fx k01) + fy((1-fx) k10 + fx k11).
__device__ __forceinline__ double bilinear64(double fx, double fy, double k00, double k01, double k10,
                                             double k11) {
  double gx = d_sub(1.0, fx), gy = d_sub(1.0, fy);
  double top = d_add(d_mul(gx, k00), d_mul(fx, k01));
  double bot = d_add(d_mul(gx, k10), d_mul(fx, k11));
  return d_add(d_mul(gy, top), d_mul(fy, bot));
}

// Vote bin of one coordinate: floor(p + sr * X + 1/2), product and sums
// each rounded once.
__device__ __forceinline__ int vote_bin64(int p, double sr, double X) {
  double a = d_add((double)p, d_mul(sr, X));
  return (int)floor(d_add(a, 0.5));
}

// Cell of one coordinate in a coarse parameter space of c = 2^lc px cells:
// floor((a + c/2) / c), a = p + sr X, the sums rounded once each and the
// division exact.
__device__ __forceinline__ int vote_cell64(int p, double sr, double X, int lc) {
  double a = d_add((double)p, d_mul(sr, X));
  return (int)floor(d_mul(d_add(a, 0.5 * (double)(1 << lc)), 1.0 / (double)(1 << lc)));
}

// ---------------------------------------------------------------------------
// double-float (hi + lo) arithmetic with explicit round-to-nearest intrinsics
// (no contraction can break the error-free transformations)
// ---------------------------------------------------------------------------
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl quick_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ dfl df_add(dfl a, dfl b) {
  dfl s = two_sum(a.hi, b.hi);
  dfl t = two_sum(a.lo, b.lo);
  s.lo = __fadd_rn(s.lo, t.hi);
  s = quick_two_sum(s.hi, s.lo);
  s.lo = __fadd_rn(s.lo, t.lo);
  return quick_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  dfl p = two_prod(a.hi, b.hi);
  p.lo = __fmaf_rn(a.hi, b.lo, p.lo);
  p.lo = __fmaf_rn(a.lo, b.hi, p.lo);
  return quick_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dfl df_sqrt(dfl a) {
  if (a.hi <= 0.0f) return {0.0f, 0.0f};
  float s = __fsqrt_rn(a.hi);
  dfl s2 = two_prod(s, s);
  float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, s2.hi), s2.lo), a.lo);
  r = __fdiv_rn(r, __fmul_rn(2.0f, s));
  return quick_two_sum(s, r);
}
__device__ __forceinline__ dfl df_div(dfl a, dfl b) {
  float q1 = __fdiv_rn(a.hi, b.hi);
  dfl p = df_mul({q1, 0.0f}, b);
  dfl r = df_add(a, {-p.hi, -p.lo});
  float q2 = __fdiv_rn(r.hi, b.hi);
  return quick_two_sum(q1, q2);
}
// exact-ish conversion of an int64 (|x| < 2^62) to double-float
__device__ __forceinline__ dfl df_from_ll(long long x) {
  float hi = __ll2float_rn(x);
  long long rem = x - (long long)hi;
  return {hi, __ll2float_rn(rem)};
}

// ---------------------------------------------------------------------------
// certified rounding of one vote coordinate
// ---------------------------------------------------------------------------
// Returns floor(t + 1/2) for t = sr * X (X = Xhi + Xlo within the bounds
// encoded in kfast, kref), or INT_MIN when double precision is needed.
// kfast: |fl(sr*Xhi) - sr*X_def| <= r*kfast + 1e-10 (X_def: the direction of
// the double-precision definition).  kref: the same after the double-float
// product.
__device__ __forceinline__ int vote_offset(float sr, float r, float xhi, float xlo, float kfast, float kref) {
  float t = __fmul_rn(sr, xhi);
  float n = floorf(__fadd_rn(t, 0.5f));
  float p = __fsub_rn(t, __fsub_rn(n, 0.5f));  // exact: distance above the lower boundary
  float m = __fmaf_rn(r, kfast, 1e-10f);
  // 1 - p is exact for p >= 1/2 (Sterbenz), so both tests compare exact
  // distances with the margin
  if (p > m && (p < 0.5f || __fsub_rn(1.0f, p) > m)) return (int)n;
  // double-float refinement: t = p2 + e2 with p2 = fl(sr*xhi) exactly split
  dfl tp = two_prod(sr, xhi);
  float e2 = __fmaf_rn(sr, xlo, tp.lo);
  float p2 = __fsub_rn(tp.hi, __fsub_rn(n, 0.5f));  // exact
  float q2 = __fsub_rn(1.0f, p2);                   // exact when p2 >= 1/2
  float mr = __fmaf_rn(r, kref, 1e-10f);
  bool low_ok = p2 > __fsub_rn(mr, e2);             // d = p2 + e2 > mr
  bool low_bad = p2 < __fsub_rn(-mr, e2);           // d < -mr
  bool up_ok = (p2 < 0.5f) || (q2 > __fadd_rn(mr, e2));   // 1 - d > mr
  bool up_bad = (p2 >= 0.5f) && (q2 < __fsub_rn(e2, mr)); // d > 1 + mr
  if (low_ok && up_ok) return (int)n;
  if (low_bad) return (int)n - 1;
  if (up_bad) return (int)n + 1;
  return INT_MIN;
}

// floor(sr X_def) with the same margins (a coarse parameter space bins votes
// by cells whose edges are at integer offsets from the pixel), or INT_MIN
// when the margins cannot decide.
__device__ __forceinline__ int vote_floor(float sr, float r, float xhi, float xlo, float kfast, float kref) {
  float t = __fmul_rn(sr, xhi);
  float n = floorf(t);
  float p = __fsub_rn(t, n);  // exact: distance above the lower boundary, in [0, 1)
  float m = __fmaf_rn(r, kfast, 1e-10f);
  if (p > m && (p < 0.5f || __fsub_rn(1.0f, p) > m)) return (int)n;
  dfl tp = two_prod(sr, xhi);
  float e2 = __fmaf_rn(sr, xlo, tp.lo);
  float p2 = __fsub_rn(tp.hi, n);  // exact
  float q2 = __fsub_rn(1.0f, p2);  // exact when p2 >= 1/2
  float mr = __fmaf_rn(r, kref, 1e-10f);
  bool low_ok = p2 > __fsub_rn(mr, e2);
  bool low_bad = p2 < __fsub_rn(-mr, e2);
  bool up_ok = (p2 < 0.5f) || (q2 > __fadd_rn(mr, e2));
  bool up_bad = (p2 >= 0.5f) && (q2 < __fsub_rn(e2, mr));
  if (low_ok && up_ok) return (int)n;
  if (low_bad) return (int)n - 1;
  if (up_bad) return (int)n + 1;
  return INT_MIN;
}

}  // namespace rd
