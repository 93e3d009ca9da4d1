// rd_api.cu -- host side of the C ABI declared in include/rd.h: parameter
// validation, the exact weight tables, device workspaces and the launch
// sequence of one rd_detect call.
//
// The tables follow the definition operation by operation (compile with
// -ffp-contract=off so that no multiply-add is fused):
//   Gaussian taps  Q_i = floor(2^19 g_i + 1/2), g_i = e_i / sum(e),
//                  e_i = exp(-(i^2) / (2 sigma sigma)), |i| <= ceil(4 sigma)
//   level weights  floor(2^16 exp(-(dy^2 + dx^2) / (2 s s)) + 1/2),
//                  s = (sig_a r + sig_b) / c, |dx|, |dy| <= ceil(3 s), with c
//                  the parameter-space cell edge in px (1 unless coarse)
//   peak threshold S > peak_frac 2 pi  <=>  N > ((peak_frac 2 pi) 2^16) r
#include "rd_internal.cuh"
#include "rd_abi_guard.h"
#include "rd.h"

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>
#include <tuple>
#include <mutex>
#include <map>


using namespace rd;

static thread_local std::string g_create_error;

struct rd_ctx {
  rd_params p;
  int max_H, max_W, max_batch;
  int device, n_sm;
  // tables
  GaussTaps taps;
  double D64;
  float invD;
  int n_levels, n_slabs, max_rw, max_qn;
  int T;  // accumulator tile edge in cells: 64, 80, 96 or 128
  int lc;  // log2 of the parameter-space cell edge in px (rd_params.coarse)
  int T_dense, max_rw_dense;  // the dense fallback kernel's tile edge and window
  int S;  // peak levels per r-slab
  std::vector<int4> h_slabs;
  // device buffers
  int4* slabs = nullptr;
  int* q_rad = nullptr;
  int* qq_off = nullptr;
  int2* qq_tab = nullptr;
  int* qp_off = nullptr;
  uint32_t* qp_tab = nullptr;
  int* fb_list = nullptr;
  int* queue = nullptr;      // K4 work queue (bin indices)
  int* queue_ctr = nullptr;  // [0] queue length, [1] head
  int* fb_count = nullptr;
  int max_qp = 4;
  unsigned long long* nthr = nullptr;
  RidgeList rl{};
  int* bin_cnt = nullptr;
  int* bin_off = nullptr;
  int* bin_fill = nullptr;
  int* cta_cnt = nullptr;  // per (frame, bin, binning CTA) entry counts; null: frames over BIN_SMEM_MAX bins
  int* block_sums = nullptr;
  long long* bin_total = nullptr;
  uint4* pool = nullptr;
  long long pool_cap = 0, n_bins_max = 0;
  int4* peaks = nullptr;
  int* peak_count = nullptr;
  int peak_cap = 4096;
  DevStats* stats = nullptr;
  // state of the last call
  cudaStream_t last_stream = nullptr;
  int last_n = 0, last_H = 0, last_W = 0;
  int32_t* dbg_acc = nullptr;
  uint32_t* dbg_sm = nullptr;
  int route_dense = 0;
  int bin_global = 0;  // rd_debug_route bit 1: binning with global counters
  // staging for rd_detect_host
  void* stage_frames = nullptr;
  rd_ring* stage_rings = nullptr;
  int* stage_counts = nullptr;
  int* stage_offsets = nullptr;
  // stage timing
  bool timing = false, timed = false;
  // feature stage: 0 directed ridges (the method), 1 directed edges (variant)
  int features = 0;
  double edge_thresh = 0.0;
  double2* e_x64 = nullptr;  // directed edges: each record's exact direction
  // soft (differentiable) path: FP64 workspaces, allocated on first use
  bool soft_ready = false;
  double *s_t0 = nullptr, *s_t1 = nullptr, *s_a = nullptr, *s_b = nullptr, *s_c = nullptr, *s_k = nullptr,
         *s_X = nullptr, *s_Y = nullptr;
  int* s_count = nullptr;
  uint32_t* s_xy = nullptr;
  uint8_t* s_flags = nullptr;
  double *s_rk = nullptr, *s_rX = nullptr, *s_rY = nullptr, *s_ra = nullptr, *s_rb = nullptr, *s_rc = nullptr,
         *s_rm = nullptr, *s_gk = nullptr, *s_gX = nullptr, *s_gY = nullptr;
  int* s_ring_off = nullptr;
  float* s_score = nullptr;
  float* s_dparams = nullptr;
  int *s_tile_off = nullptr, *s_tile_cnt = nullptr;
  // graph mode: the captured rd_detect launch sequence and the arguments it was captured with
  bool graph_on = false;
  cudaGraphExec_t gexec = nullptr;
  const void* g_args[4] = {};
  int g_shape[5] = {};
  cudaStream_t g_stream = nullptr;
  cudaEvent_t ev[RD_N_STAGES + 1] = {};
  long long dev_bytes = 0;  // device memory the context holds (its cudaMalloc total)
  std::string err;
};

// ---------------------------------------------------------------- tables
static int gaussian_radius(float sigma) { return (int)std::ceil(4.0 * (double)sigma); }

static int gaussian_taps_impl(float sigma, int32_t* taps, int cap) {
  const double s = (double)sigma;
  const int R = gaussian_radius(sigma);
  if (2 * R + 1 > cap) return -1;
  const double den = 2.0 * s * s;
  std::vector<double> e(2 * R + 1);
  double tot = 0.0;
  for (int k = 0; k <= 2 * R; ++k) {
    double i = (double)(k - R);
    e[k] = std::exp(-(i * i) / den);
  }
  for (int k = 0; k <= 2 * R; ++k) tot = tot + e[k];
  for (int k = 0; k <= 2 * R; ++k) {
    double g = e[k] / tot;
    taps[k] = (int32_t)std::floor(g * (double)(1 << GAUSS_BITS) + 0.5);
  }
  return 2 * R + 1;
}

static double level_sigma(float sig_a, float sig_b, int r) { return (double)sig_a * (double)r + (double)sig_b; }
// window half-width in cells of c px: ceil(3 sigma(r) / c)
static int level_radius(float sig_a, float sig_b, int r, int c = 1) {
  return (int)std::ceil(3.0 * (level_sigma(sig_a, sig_b, r) / (double)c));
}

// weights of level r on a grid of c-px cells: the Gaussian of sigma(r) / c
// (c a power of two, so the division is exact)
static int level_weights_impl(float sig_a, float sig_b, int r, int32_t* w, int cap, int c = 1) {
  const double sg = level_sigma(sig_a, sig_b, r) / (double)c;
  const int Rs = (int)std::ceil(3.0 * sg);
  const int Wq = 2 * Rs + 1;
  if ((long long)Wq * Wq > cap) return -1;
  const double den = 2.0 * sg * sg;
  for (int dy = -Rs; dy <= Rs; ++dy)
    for (int dx = -Rs; dx <= Rs; ++dx) {
      double fy = (double)dy, fx = (double)dx;
      double d2 = fy * fy + fx * fx;
      w[(dy + Rs) * Wq + (dx + Rs)] = (int32_t)std::floor(std::exp(-d2 / den) * (double)(1 << SMOOTH_BITS) + 0.5);
    }
  return Wq * Wq;
}

static long long peak_threshold_impl(float peak_frac, int r) {
  const double two_pi = 2.0 * M_PI;
  double thr = (((double)peak_frac * two_pi) * (double)(1 << SMOOTH_BITS)) * (double)r;
  return (long long)std::floor(thr) + 1;
}

extern "C" int rd_gaussian_taps(float sigma, int32_t* taps, int cap) {
  if (!(sigma > 0.0f) || !taps) return -1;
  return gaussian_taps_impl(sigma, taps, cap);
}
extern "C" int rd_level_weights(float sig_a, float sig_b, int r, int32_t* w, int cap) {
  if (!w || r < 1 || !(level_sigma(sig_a, sig_b, r) > 0.0)) return -1;
  return level_weights_impl(sig_a, sig_b, r, w, cap);
}
extern "C" int64_t rd_peak_threshold(float peak_frac, int r) { return peak_threshold_impl(peak_frac, r); }

// ---------------------------------------------------------------- helpers
static rd_status fail(rd_ctx* c, rd_status s, const std::string& m) {
  if (c)
    c->err = m;
  else
    g_create_error = m;
  return s;
}

static void free_all(rd_ctx* c) {
  void* ptrs[] = {c->slabs, c->q_rad, c->qq_off, c->qq_tab, c->qp_off, c->qp_tab, c->fb_list, c->fb_count, c->queue, c->queue_ctr, c->nthr, c->rl.xy, c->rl.dir, c->rl.kvote, c->rl.hess,
                  c->rl.count, c->rl.tile_off, c->rl.tile_cnt, c->bin_cnt, c->bin_off, c->bin_fill, c->cta_cnt,
                  c->block_sums, c->bin_total, c->pool, c->peaks, c->peak_count, c->stats, c->stage_frames, c->stage_rings,
                  c->stage_counts, c->stage_offsets};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  void* edge[] = {c->e_x64};
  for (void* p : edge)
    if (p) cudaFree(p);
  void* soft[] = {c->s_t0, c->s_t1, c->s_a, c->s_b, c->s_c, c->s_k, c->s_X, c->s_Y, c->s_count, c->s_xy,
                  c->s_flags, c->s_rk, c->s_rX, c->s_rY, c->s_ra, c->s_rb, c->s_rc, c->s_rm, c->s_gk, c->s_gX,
                  c->s_gY, c->s_ring_off, c->s_score, c->s_dparams, c->s_tile_off, c->s_tile_cnt};
  for (void* p : soft)
    if (p) cudaFree(p);
}

template <typename T>
static bool dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1)) == cudaSuccess;
}

// A context's allocation: counted in its device bytes.
template <typename T>
static bool dalloc(rd_ctx* c, T** p, size_t count) {
  if (!dalloc(p, count)) return false;
  c->dev_bytes += (long long)(sizeof(T) * (count ? count : 1));
  return true;
}

static std::string validate(const rd_params* p) {
  if (!p) return "params is NULL";
  if (!(p->sigma > 0.0f && p->sigma <= 4.0f)) return "sigma must be in (0, 4]";
  if (p->r_min < 2 || p->r_max < p->r_min || p->r_max > 250) return "need 2 <= r_min <= r_max <= 250";
  if (!(p->ridge_thresh <= 0.0f)) return "ridge_thresh must be <= 0";
  if (!(p->peak_frac >= 0.0f) || !std::isfinite(p->peak_frac)) return "peak_frac must be finite and >= 0";
  if (p->vote_thresh < 0 || p->vote_thresh > 65534) return "vote_thresh must be in [0, 65534]";
  if (!(p->annulus_w >= 0.0f) || p->annulus_w > 64.0f) return "annulus_w must be in [0, 64]";
  if (!(p->sig_a >= 0.0f) || !std::isfinite(p->sig_a) || !std::isfinite(p->sig_b)) return "sig_a must be >= 0";
  if (!(level_sigma(p->sig_a, p->sig_b, p->r_min - 1) > 0.0)) return "sigma(r) must be > 0 for every level";
  if (level_radius(p->sig_a, p->sig_b, p->r_max + 1) > MAX_RS) return "level smoothing radius ceil(3 sigma(r)) above 40";
  if (p->coarse != 0 && p->coarse != 1 && p->coarse != 2 && p->coarse != 4) return "coarse must be 0, 1, 2 or 4";
  if (p->coarse > 1 && (long long)p->vote_thresh * p->coarse * p->coarse > 65534)
    return "vote_thresh * coarse^2 must be at most 65534";
  return "";
}

// ---------------------------------------------------------------- C ABI
// Geometries chosen by rd_autotune, per (H, W, r_min, r_max), for this process.
namespace {
struct TuneKey {
  int H, W, r_min, r_max, coarse;
  bool operator<(const TuneKey& o) const {
    return std::tie(H, W, r_min, r_max, coarse) < std::tie(o.H, o.W, o.r_min, o.r_max, o.coarse);
  }
};
int coarse_of(const rd_params* p) { return p->coarse > 1 ? p->coarse : 1; }
std::mutex g_tune_mutex;
std::map<TuneKey, rd_geometry> g_tuned;

bool tuned_geometry(const rd_params* p, int H, int W, rd_geometry* g) {
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  auto it = g_tuned.find(TuneKey{H, W, p->r_min, p->r_max, coarse_of(p)});
  if (it == g_tuned.end()) return false;
  *g = it->second;
  return true;
}
}  // namespace

extern "C" rd_status rd_create(const rd_params* params, int max_H, int max_W, int max_batch, rd_ctx** out) {
  return rd_create_ex(params, max_H, max_W, max_batch, nullptr, out);
}

extern "C" rd_status rd_create_ex(const rd_params* params, int max_H, int max_W, int max_batch,
                                  const rd_geometry* geometry, rd_ctx** out) {
  return rd_abi::guard(&g_create_error, [&]() -> rd_status {
    if (!out) return fail(nullptr, RD_E_INVAL, "out is NULL");
    *out = nullptr;
    std::string v = validate(params);
    if (!v.empty()) return fail(nullptr, RD_E_INVAL, v);
    rd_geometry geo{0, 0};
    if (geometry) geo = *geometry;
    const bool automatic = geo.tile == 0 && geo.slab_levels == 0;
    if (!automatic && ((geo.tile != ACC_T_LARGE && geo.tile != ACC_T && geo.tile != ACC_T_MID && geo.tile != ACC_T_SMALL) ||
                       geo.slab_levels < 4 || geo.slab_levels > MAX_SLAB_LEVELS))
      return fail(nullptr, RD_E_INVAL, "geometry: tile must be 64, 80, 96 or 128 and slab_levels 4 .. 64 (or both 0)");
    if (automatic && !tuned_geometry(params, max_H, max_W, &geo)) geo = rd_geometry{0, 0};
    const int R = gaussian_radius(params->sigma);
    if (max_H < R + 4 || max_W < R + 4 || max_H < 12 || max_W < 12 || max_H > 65535 || max_W > 65535)
      return fail(nullptr, RD_E_INVAL, "frame size must be at least max(12, ceil(4 sigma) + 4) and at most 65535");
    if (max_batch < 1 || max_batch > 65535) return fail(nullptr, RD_E_INVAL, "max_batch must be in [1, 65535]");

    // Until the context is handed out, every exit (an error return or an
    // exception) frees what it holds.
    struct Owner {
      rd_ctx* c;
      ~Owner() {
        if (c) {
          free_all(c);
          delete c;
        }
      }
    } own{new rd_ctx()};
    rd_ctx* c = own.c;
    c->p = *params;
    c->p.coarse = coarse_of(params);
    c->lc = c->p.coarse == 4 ? 2 : (c->p.coarse == 2 ? 1 : 0);
    c->max_H = max_H;
    c->max_W = max_W;
    c->max_batch = max_batch;
    if (cudaGetDevice(&c->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
      return fail(nullptr, RD_E_CUDA, "no CUDA device");
    }
    // Gaussian taps and the Hessian scale D = 64 S^2
    c->taps.R = R;
    gaussian_taps_impl(params->sigma, c->taps.q, 2 * MAX_RG + 1);
    long long S = 0;
    for (int i = 0; i <= 2 * R; ++i) S += c->taps.q[i];
    c->D64 = (double)(64LL * S * S);
    c->invD = (float)(1.0 / c->D64);
    // levels, weights, thresholds
    const int lv0 = params->r_min - 1, lv1 = params->r_max + 1;
    c->n_levels = lv1 - lv0 + 1;
    std::vector<int> h_qoff(c->n_levels), h_qrad(c->n_levels);
    std::vector<int32_t> h_qtab;
    std::vector<unsigned long long> h_nthr(c->n_levels, 0);
    c->max_qn = 1;
    for (int li = 0; li < c->n_levels; ++li) {
      int r = lv0 + li;
      int Rs = level_radius(params->sig_a, params->sig_b, r, 1 << c->lc);
      int nq = (2 * Rs + 1) * (2 * Rs + 1);
      h_qoff[li] = (int)h_qtab.size();
      h_qrad[li] = Rs;
      h_qtab.resize(h_qtab.size() + nq);
      level_weights_impl(params->sig_a, params->sig_b, r, h_qtab.data() + h_qoff[li], nq, 1 << c->lc);
      h_nthr[li] = (unsigned long long)peak_threshold_impl(params->peak_frac, r);
      c->max_qn = std::max(c->max_qn, nq + (nq & 1));
    }
    // Automatic geometry: the first of 128/32, 96/12 and 64/12 whose storage
    // fits -- for 128 the sparse kernel at three CTAs per SM; always the dense
    // fallback's per-tile storage on one SM (it splits 128-pixel tiles into
    // four 64-pixel ones).  Larger tiles cast fewer halo votes per owned voxel
    // and deeper slabs recompute fewer boundary levels.
    auto dense_tile = [](int T) { return T == ACC_T_LARGE ? ACC_T_SMALL : T; };
    auto halo_of = [&](int S) {
      int mh = 0;
      for (int lo = params->r_min; lo <= params->r_max; lo += S) {
        const int hi = std::min(lo + S - 1, params->r_max);
        for (int r = lo - 1; r <= hi + 1; ++r) mh = std::max(mh, h_qrad[r - lv0] + 1);
      }
      return mh;
    };
    int qp_need = 4;
    for (int li = 0; li < c->n_levels; ++li) qp_need = std::max(qp_need, 4 * (1 + h_qrad[li] * (h_qrad[li] + 1)));
    auto fits = [&](int T, int S, bool three_per_sm) {
      const int mh = halo_of(S), Td = dense_tile(T);
      const size_t sp = sparse_smem_bytes(T + 2 * mh, qp_need);
      return vote_smem_bytes(Td + 2 * mh, Td, c->max_qn) <= 227 * 1024 && sp <= 227 * 1024 &&
             (!three_per_sm || 3 * (sp + 1024) <= 228 * 1024);
    };
    if (geo.tile == 0) {
      if (fits(ACC_T_LARGE, DEFAULT_SLAB_LEVELS, true))
        geo = rd_geometry{ACC_T_LARGE, DEFAULT_SLAB_LEVELS};
      else if (fits(ACC_T, SLAB_LEVELS, false))
        geo = rd_geometry{ACC_T, SLAB_LEVELS};
      else
        geo = rd_geometry{ACC_T_SMALL, SLAB_LEVELS};
    }
    // r-slabs of S peak levels; halo = 1 + the largest R_s of the slab's voting levels
    c->S = geo.slab_levels;
    int max_h = 0;
    for (int lo = params->r_min; lo <= params->r_max; lo += c->S) {
      int hi = std::min(lo + c->S - 1, params->r_max);
      int h = 0;
      for (int r = lo - 1; r <= hi + 1; ++r) h = std::max(h, h_qrad[r - lv0]);
      h += 1;
      c->h_slabs.push_back(make_int4(lo, hi, h, 0));
      max_h = std::max(max_h, h);
    }
    c->n_slabs = (int)c->h_slabs.size();
    c->T = geo.tile;
    c->T_dense = dense_tile(c->T);
    c->max_rw = c->T + 2 * max_h;
    c->max_rw_dense = c->T_dense + 2 * max_h;
    // per slab: (weight, offset) of every tap of its voting levels; offsets are
    // relative to the window centre in the slab's shared-memory layout
    std::vector<int> h_qqoff((size_t)c->n_slabs * (c->S + 2), 0);
    std::vector<int2> h_qqtab;
    std::vector<int> h_qpoff((size_t)c->n_slabs * (c->S + 2), 0);
    std::vector<uint32_t> h_qptab;
    for (int si = 0; si < c->n_slabs; ++si) {
      const int4 sl = c->h_slabs[si];
      const int RW = c->T + 2 * sl.z;         // the sparse kernel's slab row
      const int RWd = c->T_dense + 2 * sl.z;  // the dense kernel's slab row
      for (int r = sl.x - 1; r <= sl.y + 1; ++r) {
        const int li = r - lv0, Rs = h_qrad[li], Wq = 2 * Rs + 1;
        h_qqoff[(size_t)si * (c->S + 2) + (r - sl.x + 1)] = (int)h_qqtab.size();
        const int32_t* q = h_qtab.data() + h_qoff[li];
        for (int dy = 0; dy < Wq; ++dy)
          for (int dx = 0; dx < Wq; ++dx) h_qqtab.push_back(make_int2(q[dy * Wq + dx], (dy - Rs) * RWd + (dx - Rs)));
        if (h_qqtab.size() & 1) h_qqtab.push_back(make_int2(0, 0));  // even count: 16-byte tap pairs
        // taps for the sparse kernel in rotation orbits: Q depends on
        // dx^2 + dy^2 only, so the four taps (dx, dy), (-dy, dx), (-dx, -dy),
        // (dy, -dx) share one weight.  Entry 0 is the centre {0, 0, Q(0,0), 0};
        // then, for dx in 1..Rs and dy in 0..Rs (one tap of every orbit),
        // {o1, o2, Q, 0} with o1 = dy RW + dx and o2 = dx RW - dy: the orbit is
        // at offsets +-o1 and +-o2 from the centre.
        h_qpoff[(size_t)si * (c->S + 2) + (r - sl.x + 1)] = (int)h_qptab.size();
        auto qat = [&](int dx, int dy) { return (uint32_t)q[(dy + Rs) * Wq + (dx + Rs)]; };
        h_qptab.insert(h_qptab.end(), {0u, 0u, qat(0, 0), 0u});
        for (int dx = 1; dx <= Rs; ++dx)
          for (int dy = 0; dy <= Rs; ++dy) {
            const uint32_t w = qat(dx, dy);
            if (qat(-dy, dx) != w || qat(-dx, -dy) != w || qat(dy, -dx) != w) {
              return fail(nullptr, RD_E_INVAL, "smoothing weights are not invariant under quarter turns");
            }
            h_qptab.insert(h_qptab.end(), {(uint32_t)(dy * RW + dx), (uint32_t)(dx * RW - dy), w, 0u});
          }
        c->max_qp = std::max(c->max_qp, 4 * (1 + Rs * (Rs + 1)));
      }
    }
    if (vote_smem_bytes(c->max_rw_dense, c->T_dense, c->max_qn) > 227 * 1024 ||
        sparse_smem_bytes(c->max_rw, c->max_qp) > 227 * 1024 || c->max_rw * c->max_rw > 65535 * 2) {
      return fail(nullptr, RD_E_INVAL, "radius range and geometry need more shared memory than one SM has");
    }
    // workspaces
    const int n_stx = (max_W + ST_TW - 1) / ST_TW, n_sty = (max_H + ST_TH - 1) / ST_TH;
    const int max_Wc = ((max_W - 1) >> c->lc) + 1, max_Hc = ((max_H - 1) >> c->lc) + 1;  // cells
    const int n_atx = (max_Wc + c->T - 1) / c->T, n_aty = (max_Hc + c->T - 1) / c->T;
    c->rl.cap = std::max(4096, (int)std::min<long long>((long long)max_H * max_W / 4, 1LL << 24));
    c->rl.n_stx = n_stx;
    c->rl.n_sty = n_sty;
    const size_t nrec = (size_t)c->rl.cap * max_batch;
    c->n_bins_max = (long long)max_batch * n_atx * n_aty * c->n_slabs;
    c->pool_cap = std::min<long long>((long long)max_batch * max_H * max_W * 3, (1LL << 31) - 1);
    if (c->n_bins_max > INT_MAX / 4) {
      return fail(nullptr, RD_E_INVAL, "too many accumulator bins (frames x tiles x slabs > 2^31): lower max_batch");
    }
    // per-CTA bin counts of shared-memory binning: frames x bins x CTAs per
    // frame, at most min(BIN_GRID_MAX, ceil(8 SMs / frames)) CTAs per frame
    const long long nbf_max = (long long)n_atx * n_aty * c->n_slabs;
    const long long cta_cols = std::min<long long>((long long)BIN_GRID_MAX * max_batch, 8LL * c->n_sm + max_batch);
    const bool bin_local = nbf_max <= BIN_SMEM_MAX;
    bool ok = (!bin_local || dalloc(c, &c->cta_cnt, (size_t)(nbf_max * cta_cols))) &&
              dalloc(c, &c->slabs, c->n_slabs) && dalloc(c, &c->q_rad, c->n_levels) &&
              dalloc(c, &c->qq_off, h_qqoff.size()) && dalloc(c, &c->qq_tab, h_qqtab.size()) &&
              dalloc(c, &c->qp_off, h_qpoff.size()) && dalloc(c, &c->qp_tab, h_qptab.size()) &&
              dalloc(c, &c->fb_list, 4 * c->n_bins_max) && dalloc(c, &c->fb_count, 1) && dalloc(c, &c->queue, c->n_bins_max) &&
              dalloc(c, &c->queue_ctr, 2) &&
              dalloc(c, &c->nthr, c->n_levels) && dalloc(c, &c->rl.xy, nrec) &&
              dalloc(c, &c->rl.dir, nrec) && dalloc(c, &c->rl.kvote, nrec) && dalloc(c, &c->rl.hess, 3 * nrec) &&
              dalloc(c, &c->rl.count, max_batch) && dalloc(c, &c->rl.tile_off, (size_t)max_batch * n_stx * n_sty) &&
              dalloc(c, &c->rl.tile_cnt, (size_t)max_batch * n_stx * n_sty) && dalloc(c, &c->bin_cnt, c->n_bins_max) &&
              dalloc(c, &c->bin_off, c->n_bins_max) && dalloc(c, &c->bin_fill, c->n_bins_max) &&
              dalloc(c, &c->block_sums, (c->n_bins_max + 1023) / 1024 + 1) && dalloc(c, &c->bin_total, 1) &&
              dalloc(c, &c->pool, c->pool_cap) && dalloc(c, &c->peaks, (size_t)max_batch * c->peak_cap) &&
              dalloc(c, &c->peak_count, max_batch) && dalloc(c, &c->stats, 1) &&
              dalloc(c, (unsigned char**)&c->stage_frames, (size_t)max_batch * max_H * max_W * 2) &&
              dalloc(c, &c->stage_rings, (size_t)max_batch * c->peak_cap) && dalloc(c, &c->stage_counts, max_batch) &&
              dalloc(c, &c->stage_offsets, max_batch);
    if (!ok) {
      cudaGetLastError();
      return fail(nullptr, RD_E_NOMEM, "device allocation failed");
    }
    cudaError_t e = cudaMemcpy(c->slabs, c->h_slabs.data(), sizeof(int4) * c->n_slabs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(c->q_rad, h_qrad.data(), sizeof(int) * c->n_levels, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->qq_off, h_qqoff.data(), sizeof(int) * h_qqoff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->qq_tab, h_qqtab.data(), sizeof(int2) * h_qqtab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->qp_off, h_qpoff.data(), sizeof(int) * h_qpoff.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->qp_tab, h_qptab.data(), sizeof(uint32_t) * h_qptab.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(c->nthr, h_nthr.data(), sizeof(unsigned long long) * c->n_levels, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(c->stats, 0, sizeof(DevStats));
    if (e != cudaSuccess) {
      std::string m = std::string("table upload failed: ") + cudaGetErrorString(e);
      return fail(nullptr, RD_E_CUDA, m);
    }
    own.c = nullptr;
    *out = c;
    return RD_OK;
  });
}

// Enqueue every stage of rd_detect on the stream (the body of rd_detect, and
// what graph mode captures).
static rd_status detect_enqueue(rd_ctx* c, const void* frames_dev, int n, int H, int W, int dtype, void* stream,
                                rd_ring* rings_dev, int ring_cap, int* counts_dev, int* offsets_dev) {
  if (!frames_dev || !counts_dev || !offsets_dev || (ring_cap > 0 && !rings_dev) || ring_cap < 0)
    return fail(c, RD_E_INVAL, "NULL buffer or negative ring_cap");
  if (n < 1 || n > c->max_batch) return fail(c, RD_E_INVAL, "n must be in [1, max_batch]");
  if (H > c->max_H || W > c->max_W || H < c->taps.R + 4 || W < c->taps.R + 4 || H < 12 || W < 12)
    return fail(c, RD_E_INVAL, "frame size outside [max(12, ceil(4 sigma) + 4), rd_create maxima]");
  if (dtype != RD_U8 && dtype != RD_U16) return fail(c, RD_E_INVAL, "dtype must be RD_U8 or RD_U16");
  NvtxScope trace("rd_detect");
  cudaStream_t st = (cudaStream_t)stream;
  c->last_stream = st;
  c->last_n = n;
  c->last_H = H;
  c->last_W = W;

  const int n_stx = (W + ST_TW - 1) / ST_TW, n_sty = (H + ST_TH - 1) / ST_TH;
  const int Wc = ((W - 1) >> c->lc) + 1, Hc = ((H - 1) >> c->lc) + 1;  // parameter-space cells
  const int n_atx = (Wc + c->T - 1) / c->T, n_aty = (Hc + c->T - 1) / c->T;
  const long long n_bins = (long long)n * n_atx * n_aty * c->n_slabs;
  RidgeList rl = c->rl;
  rl.n_stx = n_stx;
  rl.n_sty = n_sty;

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) {
    if (e == cudaSuccess) e = x;
  };
  chk(cudaMemsetAsync(rl.count, 0, sizeof(int) * n, st));
  chk(cudaMemsetAsync(c->bin_cnt, 0, sizeof(int) * n_bins, st));
  chk(cudaMemsetAsync(c->bin_fill, 0, sizeof(int) * n_bins, st));
  chk(cudaMemsetAsync(c->peak_count, 0, sizeof(int) * n, st));
  chk(cudaMemsetAsync(c->stats, 0, sizeof(DevStats), st));
  chk(cudaMemsetAsync(c->fb_count, 0, sizeof(int), st));
  if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("memset: ") + cudaGetErrorString(e));

  auto mark = [&](int i) {
    if (c->timing) chk(cudaEventRecord(c->ev[i], st));
  };
  c->timed = c->timing;
  mark(0);
  StencilArgs sa{};
  sa.frames = frames_dev;
  sa.n = n;
  sa.H = H;
  sa.W = W;
  sa.taps = c->taps;
  sa.edge = 0;
  sa.tau = c->p.ridge_thresh;
  sa.tau64 = (double)c->p.ridge_thresh;
  sa.D64 = c->D64;
  sa.invD = c->invD;
  sa.rl = rl;
  sa.stats = c->stats;
  if (c->features == 1) {  // directed edges replace directed ridges: -|grad| is tested as k-
    long long S = 0;
    for (int i = 0; i <= 2 * c->taps.R; ++i) S += c->taps.q[i];
    sa.edge = 1;
    sa.tau = -(float)c->edge_thresh;
    sa.tau64 = -c->edge_thresh;
    sa.D64 = (double)(128LL * S * S);
    sa.invD = (float)(1.0 / sa.D64);
    rl.x64 = c->e_x64;  // the records keep their exact double direction
    sa.rl = rl;
    NvtxScope stage("rd_detect:edges");
    chk(launch_stencil(sa, dtype, st));
    mark(1);
    mark(2);
  } else {
    NvtxScope stage("rd_detect:ridges");
    chk(launch_stencil(sa, dtype, st));
    mark(1);
    chk(launch_refine(rl, n, c->n_sm, st));
    mark(2);
  }
  if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("stencil: ") + cudaGetErrorString(e));

  BinArgs ba;
  ba.rl = rl;
  ba.n_frames = n;
  ba.H = Hc;
  ba.W = Wc;
  ba.lc = c->lc;
  ba.inv_c = 1.0f / (float)(1 << c->lc);
  ba.n_atx = n_atx;
  ba.n_aty = n_aty;
  ba.n_slabs = c->n_slabs;
  ba.T = c->T;
  ba.slabs = c->slabs;
  ba.bin_cnt = c->bin_cnt;
  ba.bin_off = c->bin_off;
  ba.bin_fill = c->bin_fill;
  ba.cta_cnt = c->bin_global ? nullptr : c->cta_cnt;  // null: global counters (large frames, or rd_debug_route)
  ba.pool = c->pool;
  ba.pool_cap = c->pool_cap;
  ba.stats = c->stats;
  {
    NvtxScope stage("rd_detect:bins");
    chk(launch_bins(ba, c->n_sm, st, n_bins, c->block_sums, c->bin_total));
  }
  mark(3);
  if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("bins: ") + cudaGetErrorString(e));

  VoteArgs va;
  va.rl = rl;
  va.n_frames = n;
  va.H = Hc;
  va.W = Wc;
  va.lc = c->lc;
  va.n_atx = n_atx;
  va.n_aty = n_aty;
  va.n_slabs = c->n_slabs;
  va.T = c->T;
  va.slab_stride = c->S + 2;
  va.slabs = c->slabs;
  va.bin_cnt = c->bin_cnt;
  va.bin_off = c->bin_off;
  va.pool = c->pool;
  va.pool_cap = c->pool_cap;
  va.q_rad = c->q_rad;
  va.qq_off = c->qq_off;
  va.qq_tab = c->qq_tab;
  va.nthr = c->nthr;
  va.r_min = c->p.r_min;
  va.r_max = c->p.r_max;
  va.vote_thresh = c->p.vote_thresh << (2 * c->lc);  // per cell: T_int c^2
  va.peaks = c->peaks;
  va.peak_cap = c->peak_cap;
  va.peak_count = c->peak_count;
  va.stats = c->stats;
  va.D64 = c->D64;
  va.dbg_acc = c->dbg_acc;
  va.dbg_sm = c->dbg_sm;
  va.max_rw = c->max_rw;
  va.T_dense = c->T_dense;
  va.max_rw_dense = c->max_rw_dense;
  va.max_qn = c->max_qn;
  va.max_qp = c->max_qp;
  va.qp_off = c->qp_off;
  va.qp_tab = c->qp_tab;
  va.fb_list = c->fb_list;
  va.fb_count = c->fb_count;
  va.fb_cap = (int)(4 * n_bins);
  va.fb_grid = 2 * c->n_sm;
  va.queue = c->queue;
  va.n_queue = c->queue_ctr;
  va.queue_head = c->queue_ctr + 1;
  va.vote_grid = c->n_sm;  // times the resident CTAs per SM (launch_vote)
  va.route_dense = c->route_dense;
  {
    NvtxScope stage("rd_detect:vote");
    chk(launch_vote(va, n_bins, st));
  }
  mark(4);
  if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("vote: ") + cudaGetErrorString(e));

  FitArgs fa;
  fa.rl = rl;
  fa.n_frames = n;
  fa.H = H;
  fa.W = W;
  fa.peaks = c->peaks;
  fa.peak_count = c->peak_count;
  fa.peak_cap = c->peak_cap;
  fa.offsets = offsets_dev;
  fa.rings = rings_dev;
  fa.ring_cap = ring_cap;
  // a coarse peak's centre is known to within c / sqrt 2 px: the annulus widens by c - 1
  fa.w = c->p.annulus_w + (float)((1 << c->lc) - 1);
  fa.w_int = (std::floor(fa.w) == fa.w) ? 1 : 0;
  fa.stats = c->stats;
  {
    NvtxScope stage("rd_detect:fit");
    chk(launch_fit(fa, c->peaks, counts_dev, offsets_dev, st));
  }
  mark(5);
  if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("fit: ") + cudaGetErrorString(e));
  return RD_OK;
}

static void drop_graph(rd_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = nullptr;
}

extern "C" rd_status rd_detect(rd_ctx* c, const void* frames_dev, int n, int H, int W, int dtype, void* stream,
                               rd_ring* rings_dev, int ring_cap, int* counts_dev, int* offsets_dev) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    if (!c) return RD_E_INVAL;
    if (!c->graph_on) return detect_enqueue(c, frames_dev, n, H, W, dtype, stream, rings_dev, ring_cap, counts_dev,
                                            offsets_dev);
    cudaStream_t st = (cudaStream_t)stream;
    if (!st) return fail(c, RD_E_INVAL, "graph mode needs a non-default stream");
    const void* args[4] = {frames_dev, rings_dev, counts_dev, offsets_dev};
    const int shape[5] = {n, H, W, dtype, ring_cap};
    const bool same = c->gexec && st == c->g_stream && std::equal(args, args + 4, c->g_args) &&
                      std::equal(shape, shape + 5, c->g_shape);
    if (!same) {  // capture this argument set once; later identical calls replay it
      drop_graph(c);
      cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("cudaStreamBeginCapture: ") + cudaGetErrorString(e));
      const bool timing = c->timing;
      c->timing = false;
      rd_status s = detect_enqueue(c, frames_dev, n, H, W, dtype, stream, rings_dev, ring_cap, counts_dev, offsets_dev);
      c->timing = timing;
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(st, &g);
      if (s != RD_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, g, 0);
      if (g) cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        c->gexec = nullptr;
        return fail(c, RD_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
      }
      std::copy(args, args + 4, c->g_args);
      std::copy(shape, shape + 5, c->g_shape);
      c->g_stream = st;
    }
    c->last_stream = st;
    c->last_n = n;
    c->last_H = H;
    c->last_W = W;
    c->timed = false;
    cudaError_t e = cudaGraphLaunch(c->gexec, st);
    if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(e));
    return RD_OK;
  });
}

extern "C" rd_status rd_set_graph(rd_ctx* c, int on) {
  if (!c) return RD_E_INVAL;
  c->graph_on = on != 0;
  drop_graph(c);
  return RD_OK;
}

extern "C" rd_status rd_detect_host(rd_ctx* c, const void* frames_host, int n, int H, int W, int dtype, void* stream,
                                    rd_ring* rings_host, int ring_cap, int* counts_host, int* offsets_host) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    NvtxScope trace("rd_detect_host");
    if (!c) return RD_E_INVAL;
    if (!frames_host || !counts_host || !offsets_host || (ring_cap > 0 && !rings_host) || ring_cap < 0)
      return fail(c, RD_E_INVAL, "NULL buffer or negative ring_cap");
    if (n < 1 || n > c->max_batch || H < 1 || W < 1 || H > c->max_H || W > c->max_W)
      return fail(c, RD_E_INVAL, "batch or frame size above the rd_create maxima");
    if (ring_cap > c->max_batch * c->peak_cap) return fail(c, RD_E_INVAL, "ring_cap above max_batch * 4096");
    if (dtype != RD_U8 && dtype != RD_U16) return fail(c, RD_E_INVAL, "dtype must be RD_U8 or RD_U16");
    cudaStream_t st = (cudaStream_t)stream;
    size_t bytes = (size_t)n * H * W * (dtype == RD_U8 ? 1 : 2);
    cudaError_t e = cudaMemcpyAsync(c->stage_frames, frames_host, bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("frames copy: ") + cudaGetErrorString(e));
    rd_status s = rd_detect(c, c->stage_frames, n, H, W, dtype, stream, c->stage_rings, ring_cap, c->stage_counts,
                            c->stage_offsets);
    if (s != RD_OK) return s;
    e = cudaMemcpyAsync(counts_host, c->stage_counts, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(offsets_host, c->stage_offsets, sizeof(int) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && ring_cap > 0) {
      long long used = (long long)offsets_host[n - 1] + counts_host[n - 1];
      used = std::min<long long>(used, ring_cap);
      if (used > 0)
        e = cudaMemcpyAsync(rings_host, c->stage_rings, sizeof(rd_ring) * used, cudaMemcpyDeviceToHost, st);
    }
    if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
    rd_stats stats;
    return rd_get_stats(c, &stats);
  });
}

extern "C" rd_status rd_get_device_bytes(const rd_ctx* c, long long* bytes) {
  if (!c || !bytes) return RD_E_INVAL;
  *bytes = c->dev_bytes;
  return RD_OK;
}

extern "C" rd_status rd_get_stats(rd_ctx* c, rd_stats* out) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    if (!c || !out) return RD_E_INVAL;
    cudaError_t e = cudaStreamSynchronize(c->last_stream);
    DevStats d{};
    if (e == cudaSuccess) e = cudaMemcpy(&d, c->stats, sizeof(DevStats), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("stats: ") + cudaGetErrorString(e));
    out->ridge_pixels = (int64_t)d.ridge;
    out->votes = (int64_t)d.votes;
    out->peaks = (int64_t)d.peaks;
    out->exact_fallbacks = (int64_t)d.fallbacks;
    out->overflow = d.overflow;
    out->n_frames = c->last_n;
    out->hotspots = (int64_t)d.hotspots;
    out->smooth_macs = (int64_t)d.smooth_macs;
    return d.overflow ? RD_E_OVERFLOW : RD_OK;
  });
}

extern "C" rd_status rd_set_timing(rd_ctx* c, int on) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    if (!c) return RD_E_INVAL;
    if (on && !c->ev[0]) {
      for (int i = 0; i <= RD_N_STAGES; ++i)
        if (cudaEventCreate(&c->ev[i]) != cudaSuccess) return fail(c, RD_E_CUDA, "cudaEventCreate failed");
    }
    c->timing = on != 0;
    return RD_OK;
  });
}

extern "C" int rd_get_timing(rd_ctx* c, float* ms, int cap) {
  if (!c || !ms || cap < 0 || !c->timed || !c->ev[0]) return -1;
  if (cudaEventSynchronize(c->ev[RD_N_STAGES]) != cudaSuccess) return -1;
  int n = std::min(cap, RD_N_STAGES);
  for (int i = 0; i < n; ++i)
    if (cudaEventElapsedTime(&ms[i], c->ev[i], c->ev[i + 1]) != cudaSuccess) return -1;
  return n;
}

extern "C" rd_status rd_destroy(rd_ctx* c) {
  if (!c) return RD_E_INVAL;
  cudaDeviceSynchronize();
  drop_graph(c);
  for (int i = 0; i <= RD_N_STAGES; ++i)
    if (c->ev[i]) cudaEventDestroy(c->ev[i]);
  free_all(c);
  delete c;
  return RD_OK;
}

extern "C" const char* rd_last_error(const rd_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

extern "C" int rd_debug_ridges(rd_ctx* c, int f, int32_t* xy, float* dir, int64_t* hess, int cap) {
  return rd_abi::guard_count(c ? &c->err : &g_create_error, [&]() -> int {
    if (!c || f < 0 || f >= c->last_n || cap < 0) return -1;
    if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) return -1;
    int cnt = 0;
    if (cudaMemcpy(&cnt, c->rl.count + f, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    int n = std::min(std::min(cnt, c->rl.cap), cap);
    size_t base = (size_t)f * c->rl.cap;
    if (n > 0) {
      std::vector<uint32_t> hxy(n);
      std::vector<float4> hdir(n);
      if (cudaMemcpy(hxy.data(), c->rl.xy + base, 4 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
      if (cudaMemcpy(hdir.data(), c->rl.dir + base, 16 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
      for (int i = 0; i < n; ++i) {
        if (xy) {
          xy[2 * i] = (int32_t)(hxy[i] & 0xffffu);
          xy[2 * i + 1] = (int32_t)(hxy[i] >> 16);
        }
        if (dir) {
          dir[2 * i] = hdir[i].x;
          dir[2 * i + 1] = hdir[i].y;
        }
      }
      if (hess && cudaMemcpy(hess, c->rl.hess + 3 * base, 24 * (size_t)n, cudaMemcpyDeviceToHost) != cudaSuccess)
        return -1;
    }
    return cnt;
  });
}

extern "C" rd_status rd_debug_route(rd_ctx* c, int flags) {
  if (!c || (flags & ~3)) return RD_E_INVAL;
  c->route_dense = flags & 1;
  c->bin_global = (flags >> 1) & 1;
  drop_graph(c);
  return RD_OK;
}

extern "C" rd_status rd_debug_capture(rd_ctx* c, int32_t* acc_dev, uint32_t* sm_dev) {
  if (!c) return RD_E_INVAL;
  c->dbg_acc = acc_dev;
  c->dbg_sm = acc_dev ? sm_dev : nullptr;
  drop_graph(c);
  return RD_OK;
}

extern "C" rd_status rd_get_geometry(const rd_ctx* c, rd_geometry* out) {
  if (!c || !out) return RD_E_INVAL;
  out->tile = c->T;
  out->slab_levels = c->S;
  return RD_OK;
}

// Autotuner: every candidate geometry runs the caller's frames through a
// temporary context (one warm-up call, two timed calls, CUDA events on the
// caller's stream); the fastest is returned and cached for rd_create.
extern "C" rd_status rd_autotune(const rd_params* params, const void* frames_dev, int n, int H, int W, int dtype,
                                 void* stream, rd_geometry* best) {
  return rd_abi::guard(&g_create_error, [&]() -> rd_status {
    NvtxScope trace("rd_autotune");
    if (!params || !frames_dev || !best || n < 1 || n > 65535)
      return fail(nullptr, RD_E_INVAL, "rd_autotune: NULL argument or n outside [1, 65535]");
    std::string v = validate(params);
    if (!v.empty()) return fail(nullptr, RD_E_INVAL, v);
    cudaStream_t st = (cudaStream_t)stream;
    const int ring_cap = n * 4096;
    rd_ring* rings = nullptr;
    int* counts = nullptr;
    int* offs = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rd_status res = RD_OK;
    if (!dalloc(&rings, (size_t)ring_cap) || !dalloc(&counts, (size_t)n) || !dalloc(&offs, (size_t)n)) {
      res = fail(nullptr, RD_E_NOMEM, "rd_autotune: output buffers");
    } else if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
      res = fail(nullptr, RD_E_CUDA, "rd_autotune: cudaEventCreate");
    }
    float best_ms = 0.0f;
    rd_geometry bg{0, 0};
    rd_status last = RD_E_NOMEM;
    std::string last_msg = "no candidate geometry could allocate its workspaces";
    const int tiles[4] = {ACC_T_SMALL, ACC_T_MID, ACC_T, ACC_T_LARGE};
    const int slabs[4] = {8, 16, 24, 32};
    for (int ti = 0; ti < 4 && res == RD_OK; ++ti)
      for (int si = 0; si < 4 && res == RD_OK; ++si) {
        const rd_geometry g{tiles[ti], slabs[si]};
        rd_ctx* c = nullptr;
        rd_status s = rd_create_ex(params, H, W, n, &g, &c);
        if (s != RD_OK) {  // does not fit this radius range, or no memory: skip
          last = s;
          last_msg = g_create_error;
          continue;
        }
        float ms = 0.0f;
        s = rd_detect(c, frames_dev, n, H, W, dtype, stream, rings, ring_cap, counts, offs);
        if (s == RD_OK && cudaEventRecord(e0, st) == cudaSuccess) {
          for (int k = 0; k < 2 && s == RD_OK; ++k) s = rd_detect(c, frames_dev, n, H, W, dtype, stream, rings, ring_cap, counts, offs);
          if (s == RD_OK && (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
            s = RD_E_CUDA;
        }
        if (s != RD_OK) {
          res = fail(nullptr, s, std::string("rd_autotune: ") + c->err);
          rd_destroy(c);
          break;
        }
        rd_destroy(c);
        if (bg.tile == 0 || ms < best_ms) {
          best_ms = ms;
          bg = g;
        }
      }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(rings);
    cudaFree(counts);
    cudaFree(offs);
    if (res != RD_OK) return res;
    if (bg.tile == 0) return fail(nullptr, last, "rd_autotune: " + last_msg);
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      g_tuned[TuneKey{H, W, params->r_min, params->r_max, coarse_of(params)}] = bg;
    }
    *best = bg;
    return RD_OK;
  });
}


// ---------------------------------------------------------------- soft (differentiable) path
static rd_status ensure_soft(rd_ctx* c) {
  if (c->soft_ready) return RD_OK;
  const size_t px = (size_t)c->max_batch * c->max_H * c->max_W;
  const size_t rec = (size_t)c->max_batch * c->rl.cap;
  const size_t rings = (size_t)c->max_batch * c->peak_cap;
  bool ok = dalloc(c, &c->s_t0, px) && dalloc(c, &c->s_t1, px) && dalloc(c, &c->s_a, px) && dalloc(c, &c->s_b, px) &&
            dalloc(c, &c->s_c, px) && dalloc(c, &c->s_k, px) && dalloc(c, &c->s_X, px) && dalloc(c, &c->s_Y, px) &&
            dalloc(c, &c->s_count, c->max_batch) && dalloc(c, &c->s_xy, rec) && dalloc(c, &c->s_flags, rec) &&
            dalloc(c, &c->s_rk, rec) && dalloc(c, &c->s_rX, rec) && dalloc(c, &c->s_rY, rec) && dalloc(c, &c->s_ra, rec) &&
            dalloc(c, &c->s_rb, rec) && dalloc(c, &c->s_rc, rec) && dalloc(c, &c->s_rm, rec) && dalloc(c, &c->s_gk, rec) &&
            dalloc(c, &c->s_gX, rec) && dalloc(c, &c->s_gY, rec) && dalloc(c, &c->s_ring_off, (size_t)c->max_batch + 1) &&
            dalloc(c, &c->s_score, rings) && dalloc(c, &c->s_dparams, 3 * rings) &&
            dalloc(c, &c->s_tile_off, (size_t)c->max_batch * ((c->max_W + 31) / 32) * ((c->max_H + 31) / 32)) &&
            dalloc(c, &c->s_tile_cnt, (size_t)c->max_batch * ((c->max_W + 31) / 32) * ((c->max_H + 31) / 32));
  if (!ok) {
    cudaGetLastError();
    return fail(c, RD_E_NOMEM, "soft path: device allocation failed");
  }
  c->soft_ready = true;
  return RD_OK;
}

// Validate, allocate on first use and enqueue the soft stencil stage (Gaussian,
// Hessian, eigen, ridge records) of n frames; fills *a.
static rd_status soft_prepare(rd_ctx* c, const void* frames, int n, int H, int W, int dtype, cudaStream_t st,
                              const rd_ring* rings, const int* counts, SoftArgs* a) {
  if (!frames || !rings || !counts) return fail(c, RD_E_INVAL, "NULL argument");
  if (n < 1 || n > c->max_batch) return fail(c, RD_E_INVAL, "n must be in [1, max_batch]");
  if (H > c->max_H || W > c->max_W || H < c->taps.R + 4 || W < c->taps.R + 4 || H < 12 || W < 12)
    return fail(c, RD_E_INVAL, "frame size outside [max(12, ceil(4 sigma) + 4), rd_create maxima]");
  if (dtype != RD_U8 && dtype != RD_U16 && dtype != RD_F32)
    return fail(c, RD_E_INVAL, "dtype must be RD_U8, RD_U16 or RD_F32");
  rd_status s = ensure_soft(c);
  if (s != RD_OK) return s;
  *a = SoftArgs{};
  a->frames = frames;
  a->dtype = dtype;
  a->n = n;
  a->H = H;
  a->W = W;
  a->R = c->taps.R;
  long long S = 0;
  for (int i = 0; i <= 2 * c->taps.R; ++i) S += c->taps.q[i];
  for (int i = 0; i <= 2 * c->taps.R; ++i) a->g[i] = (double)c->taps.q[i] / (double)S;
  a->tau = (double)c->p.ridge_thresh;
  a->temp = std::max(std::fabs(a->tau), 1e-6) / 4.0;
  a->sig_a = (double)c->p.sig_a;
  a->sig_b = (double)c->p.sig_b;
  a->sig_ann = 0.5 * (double)c->p.annulus_w;
  a->t0 = c->s_t0;
  a->t1 = c->s_t1;
  a->a = c->s_a;
  a->b = c->s_b;
  a->c = c->s_c;
  a->k = c->s_k;
  a->X = c->s_X;
  a->Y = c->s_Y;
  a->cap = c->rl.cap;
  a->count = c->s_count;
  a->n_tx = (W + 31) / 32;
  a->n_ty = (H + 31) / 32;
  a->tile_off = c->s_tile_off;
  a->tile_cnt = c->s_tile_cnt;
  a->xy = c->s_xy;
  a->flags = c->s_flags;
  a->rk = c->s_rk;
  a->rX = c->s_rX;
  a->rY = c->s_rY;
  a->ra = c->s_ra;
  a->rb = c->s_rb;
  a->rc = c->s_rc;
  a->rm = c->s_rm;
  a->gk = c->s_gk;
  a->gX = c->s_gX;
  a->gY = c->s_gY;
  a->rings = rings;
  a->ring_off = c->s_ring_off;
  a->max_rings = INT_MAX;
  c->last_stream = st;
  cudaError_t e = cudaMemsetAsync(c->s_count, 0, sizeof(int) * n, st);
  if (e == cudaSuccess) e = launch_soft_stencil(*a, st);
  if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("soft stencil: ") + cudaGetErrorString(e));
  return RD_OK;
}

extern "C" rd_status rd_soft_score(rd_ctx* c, const void* frames_dev, int n, int H, int W, int dtype, void* stream,
                                   const rd_ring* rings_dev, const int* counts_dev, float* score_dev,
                                   float* dparams_dev) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    NvtxScope trace("rd_soft_score");
    if (!c) return RD_E_INVAL;
    if (!score_dev) return fail(c, RD_E_INVAL, "score_dev is NULL");
    cudaStream_t st = (cudaStream_t)stream;
    SoftArgs a;
    rd_status s = soft_prepare(c, frames_dev, n, H, W, dtype, st, rings_dev, counts_dev, &a);
    if (s != RD_OK) return s;
    a.score = score_dev;
    a.dparams = dparams_dev;
    cudaError_t e = launch_soft_score(a, counts_dev, c->s_ring_off, st);
    if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("soft score: ") + cudaGetErrorString(e));
    return RD_OK;
  });
}

extern "C" rd_status rd_backward(rd_ctx* c, const float* frames_dev, int n, int H, int W, void* stream,
                                 const rd_ring* rings_dev, const int* counts_dev, const float* dscore_dev,
                                 float* dimage_dev, float* dparams_dev) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    NvtxScope trace("rd_backward");
    if (!c) return RD_E_INVAL;
    if (!dscore_dev || !dimage_dev) return fail(c, RD_E_INVAL, "dscore_dev and dimage_dev must not be NULL");
    cudaStream_t st = (cudaStream_t)stream;
    SoftArgs a;
    rd_status s = soft_prepare(c, frames_dev, n, H, W, RD_F32, st, rings_dev, counts_dev, &a);
    if (s != RD_OK) return s;
    const size_t rec = sizeof(double) * (size_t)n * c->rl.cap;
    cudaError_t e = cudaMemsetAsync(c->s_gk, 0, rec, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->s_gX, 0, rec, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->s_gY, 0, rec, st);
    a.dscore = dscore_dev;
    a.dparams = dparams_dev;
    a.accumulate = 1;
    a.dimage = dimage_dev;
    if (e == cudaSuccess) e = launch_soft_score(a, counts_dev, c->s_ring_off, st);
    if (e == cudaSuccess) e = launch_soft_backward_image(a, st);
    if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("soft backward: ") + cudaGetErrorString(e));
    return RD_OK;
  });
}

extern "C" rd_status rd_refine(rd_ctx* c, const void* frames_dev, int n, int H, int W, int dtype, void* stream,
                               rd_ring* rings_dev, const int* counts_dev, int iters, float step) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    NvtxScope trace("rd_refine");
    if (!c) return RD_E_INVAL;
    if (iters < 0 || !(step > 0.0f)) return fail(c, RD_E_INVAL, "iters must be >= 0 and step > 0");
    cudaStream_t st = (cudaStream_t)stream;
    SoftArgs a;
    rd_status s = soft_prepare(c, frames_dev, n, H, W, dtype, st, rings_dev, counts_dev, &a);
    if (s != RD_OK) return s;
    a.rings_mut = rings_dev;
    a.score = c->s_score;
    a.dparams = c->s_dparams;
    a.max_rings = c->max_batch * c->peak_cap;
    a.step = step;
    cudaError_t e = cudaSuccess;
    for (int it = 0; it < iters && e == cudaSuccess; ++it) {
      e = launch_soft_score(a, counts_dev, c->s_ring_off, st);
      if (e == cudaSuccess) e = launch_soft_refine_step(a, st);
    }
    if (e != cudaSuccess) return fail(c, RD_E_CUDA, std::string("refine: ") + cudaGetErrorString(e));
    return RD_OK;
  });
}


// ---------------------------------------------------------------- feature stage
extern "C" rd_status rd_set_features(rd_ctx* c, int features, float edge_thresh) {
  return rd_abi::guard(c ? &c->err : &g_create_error, [&]() -> rd_status {
    if (!c) return RD_E_INVAL;
    if (features != RD_FEATURES_RIDGE && features != RD_FEATURES_EDGE)
      return fail(c, RD_E_INVAL, "features must be RD_FEATURES_RIDGE or RD_FEATURES_EDGE");
    if (!(edge_thresh >= 0.0f) || !std::isfinite(edge_thresh)) return fail(c, RD_E_INVAL, "edge_thresh must be >= 0");
    if (features == RD_FEATURES_EDGE && !c->e_x64) {
      const size_t rec = (size_t)c->max_batch * c->rl.cap;
      bool ok = dalloc(c, &c->e_x64, rec);
      if (!ok) {
        cudaGetLastError();
        return fail(c, RD_E_NOMEM, "edge workspaces: device allocation failed");
      }
    }
    c->features = features;
    c->edge_thresh = (double)edge_thresh;
    drop_graph(c);
    return RD_OK;
  });
}
