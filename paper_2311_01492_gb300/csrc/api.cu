// C ABI of libasora: handles, validation, memory, launches (see include/asora.h).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <unordered_map>

#include "asora_internal.cuh"

namespace asora {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---------------------------------------------------------- device memory
static std::mutex g_mem_mutex;
static std::unordered_map<void*, size_t> g_mem_sizes;
static int64_t g_mem_live = 0;
static int64_t g_mem_limit = -1;  // -1: not read yet, 0: no limit

static int64_t mem_limit_locked() {
  if (g_mem_limit < 0) {
    g_mem_limit = 0;
    if (const char* v = std::getenv("ASORA_DEVICE_MEMORY_LIMIT")) {
      char* end = nullptr;
      const long long x = std::strtoll(v, &end, 10);
      if (end != v && x > 0) g_mem_limit = x;
    }
  }
  return g_mem_limit;
}

cudaError_t dev_malloc_raw(void** p, size_t bytes) {
  *p = nullptr;
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  const int64_t lim = mem_limit_locked();
  if (lim > 0 && g_mem_live + (int64_t)bytes > lim) return cudaErrorMemoryAllocation;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return e;
  }
  g_mem_sizes[*p] = bytes;
  g_mem_live += (int64_t)bytes;
  return cudaSuccess;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  {
    std::lock_guard<std::mutex> lk(g_mem_mutex);
    auto it = g_mem_sizes.find(p);
    if (it != g_mem_sizes.end()) {
      g_mem_live -= (int64_t)it->second;
      g_mem_sizes.erase(it);
    }
  }
  return cudaFree(p);
}

rt_status fail(rt_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

rt_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a sticky-free error so the next call starts clean
  return e == cudaErrorMemoryAllocation ? RT_ERR_OOM : RT_ERR_CUDA;
}

static int isqrt_h(int64_t x) {
  if (x <= 0) return 0;
  int64_t r = (int64_t)std::sqrt((double)x);
  while (r * r > x) --r;
  while ((r + 1) * (r + 1) <= x) ++r;
  return (int)r;
}

static void free_grid(Grid* g) {
  dev_free(g->boxes_d); dev_free(g->gtab); dev_free(g->htab);
  dev_free(g->dtau); dev_free(g->dtauT); dev_free(g->invn);
  free_sources(*g);
  dev_free(g->geo); dev_free(g->georow); dev_free(g->queue); dev_free(g->err);
  dev_free(g->cube); dev_free(g->unconv); dev_free(g->xbuf); dev_free(g->xavg);
  dev_free(g->xavg2); dev_free(g->xhi_int); dev_free(g->flags); dev_free(g->counters);
  dev_free(g->bwd_stack); dev_free(g->dq_merged);
  free_row_tables(*g);
  if (g->it_exec) cudaGraphExecDestroy(g->it_exec);
  if (g->it_stream) cudaStreamDestroy(g->it_stream);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
}

#define TRY(x)                                      \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x); \
  } while (0)

// Cell-size dependent constants of a box record.
static void set_box_cell(BoxDev& B, double c, double sigma0) {
  B.cell = c;
  B.inv_cell3 = 1.0 / (c * c * c);
  B.thin_fac = sigma0 / (c * c);
  B.sig_cell = sigma0 * c;
}

static rt_status ensure_geometry(Grid& g, int mmax) {
  if (mmax <= g.geo_mmax) return RT_OK;
  GeoEntry* geo = nullptr;
  GeoRow* georow = nullptr;
  TRY(dev_malloc(&geo, geo_count(mmax) * sizeof(GeoEntry)));
  cudaError_t e = dev_malloc(&georow, georow_count(mmax) * sizeof(GeoRow));
  if (e == cudaSuccess) e = launch_geometry(geo, georow, mmax, g.stream);
  if (e != cudaSuccess) {
    dev_free(geo);
    dev_free(georow);
    return cuda_fail(e, "geometry");
  }
  dev_free(g.geo);
  dev_free(g.georow);
  g.geo = geo;
  g.georow = georow;
  g.geo_mmax = mmax;
  return RT_OK;
}

// Largest layer half-width min(m, floor(sqrt(r2 - m^2))) over the layers of a face.
static int face_hcap(int r2, int nmax) {
  int h = 1;
  const int L = std::min(isqrt_h(r2), nmax / 2 + 1);
  for (int m = 1; m <= L; ++m) h = std::max(h, std::min(m, isqrt_h((int64_t)r2 - (int64_t)m * m)));
  return h;
}

static TraceArgs base_args(Grid& g) {
  TraceArgs a{};
  a.boxes = g.boxes_d;
  a.dtau = g.dtau;
  a.dtauT = g.dtauT;
  a.invn = g.invn;
  a.src = g.src;
  a.ndot = g.ndot;
  a.r2lim = g.r2lim;
  a.queue = g.queue;
  a.geo = g.geo;
  a.georow = g.georow;
  a.rtab = g.rtab;
  a.rtab_off = g.rtab_off;
  a.rtab_first = g.rtab_first;
  a.rtab_hcap = g.rtab_hcap;
  a.rtab_slot = g.rtab_slot;
  a.rtab_max_r2 = g.rtab_max_r2;
  a.itab = g.itab;
  a.itab_off = g.itab_off;
  a.neg_zero = -0.0;
  a.interp_mode = g.interp_mode;
  a.tau_w0 = g.tau_w0;
  a.geo_mmax = g.geo_mmax;
  a.tab.g = g.gtab;
  a.tab.h = g.htab;
  a.tab.kind = g.tab_kind;
  a.tab.E0 = g.E0;
  a.tab.B = g.B;
  if (g.tab_kind == RT_TABLE_GREY_EXACT) {
    // exp(-tau) is exactly 0 in double beyond tau = 746; skip the rate there
    const double lim = 750.0;
    std::memcpy(&a.tab.tau_max_bits, &lim, 8);
    a.tab.tau_min_bits = 0;
  } else {
    const double tmin = std::ldexp(1.0, -g.E0), tmax = std::ldexp(1.0, g.E1);
    std::memcpy(&a.tab.tau_min_bits, &tmin, 8);
    std::memcpy(&a.tab.tau_max_bits, &tmax, 8);
  }
  a.tau_lim = g.p.tau_lim;
  a.sigma0 = g.p.sigma0_cm2;
  a.err = g.err;
  a.rate_cells = g.counters;
  {
    double tmax;
    std::memcpy(&tmax, &a.tab.tau_max_bits, 8);
    const double bound = tmax * (1.0 + std::ldexp(1.0, -40));
    std::memcpy(&a.exit_bits, &bound, 8);
  }
  a.early_exit = 0;
  return a;
}

// Error bits latched by the kernels since the last check (the caller has
// synchronised the grid's stream); clears them.
static rt_status latched_errors(Grid& g) {
  int herr = 0;
  TRY(cudaMemcpy(&herr, g.err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!herr) return RT_OK;
  TRY(cudaMemset(g.err, 0, sizeof(int)));
  std::string what;
  if (herr & ERR_LAYER_CAP) what += " layer wider than the shared-memory capacity;";
  if (herr & ERR_GEO) what += " layer beyond the geometry table;";
  if (herr & ERR_CUBE) what += " source extent beyond the plain schedule's cube;";
  if (herr & ERR_INPUT) what += " invalid input data;";
  return fail(RT_ERR_BOUNDS, "device-side check failed (error bits " + std::to_string(herr) +
                                 "):" + what + " the results of the last trace are incomplete");
}

static rt_status check_ready(Grid& g, const char* who) {
  if (!g.have_tables) return fail(RT_ERR_STATE, std::string(who) + ": rt_set_tables not called");
  if (!g.nH) return fail(RT_ERR_STATE, std::string(who) + ": rt_set_density not called");
  if (!g.xHI) return fail(RT_ERR_STATE, std::string(who) + ": rt_set_xHI not called");
  return RT_OK;
}

// Trace all sources, adding rates into `gamma` (already zeroed) or writing one
// source's column densities.  `items`/`n_items` select the work.
// single_r2 >= 0: the items are the 24 of one source with that R^2 limit (else
// the grid's LPT list, whose limits are g.r2_sorted_h).
static rt_status run_trace(Grid& g, double* gamma, double* coldens, const int* items, int n_items,
                           int schedule, int nsrc_plain, const int* skip = nullptr,
                           bool early_exit = false, int single_r2 = -1) {
  TraceArgs a = base_args(g);
  a.gamma = gamma;
  a.coldens = coldens;
  a.skip = skip;
  a.early_exit = early_exit ? 1 : 0;
  g.stats.launches = 0;
  TRY(cudaMemsetAsync(g.counters, 0, sizeof(unsigned long long), g.stream));
  if (schedule == RT_SCHED_PLAIN) {
    const int E = std::max(1, std::min(isqrt_h(g.max_r2), g.nmax / 2));
    const int block = 256;
    int grid = std::min(nsrc_plain, std::max(1, shells_max_grid(block)));
    const size_t side = 2 * (size_t)E + 1;
    const size_t need = side * side * side * sizeof(double) * (size_t)grid;
    if (need > g.cube_bytes) {
      dev_free(g.cube);
      g.cube = nullptr;
      g.cube_bytes = 0;
      TRY(dev_malloc(&g.cube, need));
      g.cube_bytes = need;
    }
    a.scratch = g.cube;
    a.hcap = E;
    a.items = items;
    a.n_items = nsrc_plain;
    TRY(cudaMemsetAsync(g.queue, 0, sizeof(int), g.stream));
    TRY(launch_trace_shells(g, a, block, grid));
    g.stats.block = block;
    g.stats.grid = grid;
    g.stats.launches = 1;
    g.stats.items = nsrc_plain;
  } else {
    if (g.nmax > 1290)
      return fail(RT_ERR_INVALID, "rt_raytrace: the batched schedule needs boxes of at most "
                                  "1290^3 cells (32-bit offsets); use RT_SCHED_PLAIN");
    // Batched: items of large sources are traced by whole CTAs, items whose
    // layers fit g.hsmall by single warps, and the faces of sources whose layers
    // fit g.hface by single warps that trace a face whole.  Items come
    // in LPT order (24 per source, r2 non-increasing), so each mode gets a
    // contiguous range of sources: [0, pw) CTAs, [pw, p4) warps, [p4, ns) whole faces.
    const int* r2s = single_r2 >= 0 ? &single_r2 : g.r2_sorted_h.data();
    const int ns = n_items / 24;
    auto first_fitting = [&](int hlim) {  // first source whose layers fit hlim (ns: none)
      if (hlim <= 0) return ns;
      int lo = 0, hi = ns;
      while (lo < hi) {
        const int mid = (lo + hi) / 2;
        if (face_hcap(r2s[mid], g.nmax) <= hlim) hi = mid; else lo = mid + 1;
      }
      return lo;
    };
    const int pw = first_fitting(g.hsmall);
    const int p4 = std::max(pw, first_fitting(g.hface));
    const int hbig = face_hcap(r2s[0], g.nmax);
    const bool od = a.interp_mode == RT_INTERP_OPTICAL_DEPTH;
    TRY(cudaMemsetAsync(g.queue, 0, 3 * sizeof(int), g.stream));
    a.items = items;
    g.stats.launches = 0;
    // warp modes: CTAs of 1..8 warps, whichever keeps the most warps resident (a
    // warp's shared memory grows with its layer capacity, and every CTA also
    // reserves some; ties go to the larger CTA)
    auto warp_launch = [&](int mode, int hcap, int item_begin, int item_end, int* queue) {
      int wpb = 8, maxg = 0;
      for (int cand = 8; cand >= 1; --cand) {
        const int mg = faces_max_grid(mode, faces_smem_bytes(hcap, mode, od) * cand, cand, od);
        if (mg * cand > maxg * wpb) {
          maxg = mg;
          wpb = cand;
        }
      }
      if (maxg <= 0) return fail(RT_ERR_CUDA, "rt_raytrace: no occupancy for a warp face kernel");
      g.warps_per_block = wpb;
      TraceArgs b = a;
      b.hcap = hcap;
      b.item_begin = item_begin;
      b.n_items = item_end;
      b.queue = queue;
      const int nitem = item_end - item_begin;
      const int grid = std::max(1, std::min((nitem + wpb - 1) / wpb, maxg));
      TRY(launch_trace_faces(g, b, mode, grid, faces_smem_bytes(hcap, mode, od) * wpb, wpb));
      g.stats.launches += 1;
      if (g.stats.launches == 1) {
        g.stats.block = 32 * wpb;
        g.stats.grid = grid;
      }
      return RT_OK;
    };
    if (pw > 0) {
      const int block = g.block_big;
      const size_t smem = faces_smem_bytes(hbig, block, od);
      if (smem > 227 * 1024)
        return fail(RT_ERR_INVALID, "rt_raytrace: radius too large for the batched schedule's "
                                    "shared-memory layers; use RT_SCHED_PLAIN");
      const int maxg = faces_max_grid(block, smem, 8, od);
      if (maxg <= 0) return fail(RT_ERR_CUDA, "rt_raytrace: no occupancy for the face kernel");
      TraceArgs b = a;
      b.hcap = hbig;
      b.item_begin = 0;
      b.n_items = 24 * pw;
      b.queue = g.queue;
      const int grid = std::max(1, std::min(b.n_items, maxg));
      TRY(launch_trace_faces(g, b, block, grid, smem));
      g.stats.block = block;
      g.stats.grid = grid;
      g.stats.launches += 1;
    }
    if (p4 > pw) {
      rt_status ws = warp_launch(32, face_hcap(r2s[pw], g.nmax), 24 * pw, 24 * p4, g.queue + 1);
      if (ws != RT_OK) return ws;
    }
    if (ns > p4) {  // whole faces: face items it -> items[4 it]
      rt_status ws = warp_launch(4, face_hcap(r2s[p4], g.nmax), 6 * p4, 6 * ns, g.queue + 2);
      if (ws != RT_OK) return ws;
    }
    g.stats.items = n_items;
  }
  g.stats.schedule = schedule;
  return RT_OK;
}

}  // namespace asora

using namespace asora;

extern "C" {

void rt_params_default(rt_params* p) {
  if (!p) return;
  p->sigma0_cm2 = 6.30e-18;
  p->tau_lim = 1e-7;
}

const char* rt_last_error(void) { return g_last_error.c_str(); }

long long rt_kernel_launch_count(void) { return g_launches.load(); }

rt_status rt_ensemble_create(rt_grid_t* out, int nbox, const int* h_n, const double* h_cell_cm,
                             const rt_params* p, rt_stream_t s) {
  if (!out) return fail(RT_ERR_INVALID, "rt_ensemble_create: null handle pointer");
  *out = nullptr;
  if (nbox < 1 || nbox > (1 << 20) || !h_n || !h_cell_cm)
    return fail(RT_ERR_INVALID, "rt_ensemble_create: bad box list");
  rt_params prm;
  rt_params_default(&prm);
  if (p) prm = *p;
  if (!(prm.sigma0_cm2 > 0) || !std::isfinite(prm.sigma0_cm2) || !(prm.tau_lim >= 0) ||
      !std::isfinite(prm.tau_lim))
    return fail(RT_ERR_INVALID, "rt_ensemble_create: bad parameters");
  Grid* g = new Grid;
  g->p = prm;
  g->stream = (cudaStream_t)s;
  g->nbox = nbox;
  int64_t off = 0;
  for (int b = 0; b < nbox; ++b) {
    const int n = h_n[b];
    const double c = h_cell_cm[b];
    if (n < 1 || n > 4096 || !(c > 0) || !std::isfinite(c)) {
      delete g;
      return fail(RT_ERR_INVALID, "rt_ensemble_create: box size must be 1..4096 and cell > 0");
    }
    BoxDev B;
    B.n = n;
    B.wlo = -(n / 2);
    B.whi = (n % 2 == 0) ? n / 2 - 1 : n / 2;
    B.off = off;
    set_box_cell(B, c, prm.sigma0_cm2);
    g->boxes_h.push_back(B);
    g->cell_comoving.push_back(c);
    off += (int64_t)n * n * n;
    g->nmax = std::max(g->nmax, n);
  }
  g->ncell = off;
  cudaError_t e = cudaSuccess;
  e = dev_malloc(&g->boxes_d, nbox * sizeof(BoxDev));
  if (e == cudaSuccess) e = cudaMemcpy(g->boxes_d, g->boxes_h.data(), nbox * sizeof(BoxDev), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = dev_malloc(&g->dtau, g->ncell * sizeof(double));
  if (e == cudaSuccess) e = dev_malloc(&g->dtauT, g->ncell * sizeof(double));
  if (e == cudaSuccess) e = dev_malloc(&g->invn, g->ncell * sizeof(double));
  if (e == cudaSuccess) e = dev_malloc(&g->queue, 64 * sizeof(int));
  if (e == cudaSuccess) e = dev_malloc(&g->err, 2 * sizeof(int));  // [0] traces, [1] validation
  if (e == cudaSuccess) e = cudaMemset(g->err, 0, 2 * sizeof(int));
  if (e == cudaSuccess) e = dev_malloc(&g->unconv, 16 * sizeof(int64_t));
  if (e == cudaSuccess) e = dev_malloc(&g->flags, 16 * sizeof(int));
  if (e == cudaSuccess) e = dev_malloc(&g->counters, 8 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(g->counters, 0, 8 * sizeof(unsigned long long));
  for (auto& ev : g->ev)
    if (e == cudaSuccess) e = cudaEventCreate(&ev);
  if (e != cudaSuccess) {
    rt_status st = cuda_fail(e, "rt_ensemble_create");
    free_grid(g);
    return st;
  }
  *out = reinterpret_cast<rt_grid_t>(g);
  return RT_OK;
}

rt_status rt_grid_create(rt_grid_t* out, int n, double cell_cm, const rt_params* p, rt_stream_t s) {
  return rt_ensemble_create(out, 1, &n, &cell_cm, p, s);
}

rt_status rt_set_stream(rt_grid_t h, rt_stream_t s) {
  if (!h) return fail(RT_ERR_INVALID, "rt_set_stream: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  g.stream = (cudaStream_t)s;
  ++g.epoch;
  return RT_OK;
}

rt_status rt_set_tables(rt_grid_t h, int kind, int E0, int E1, int bits, const double* h_g,
                        const double* h_h) {
  if (!h) return fail(RT_ERR_INVALID, "rt_set_tables: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  const int K = rt_table_nknots(E0, E1, bits);
  if (K < 0 || E0 > 1000 || E1 > 1000 || bits > 10)
    return fail(RT_ERR_INVALID, "rt_set_tables: need 1 <= E0,E1 <= 1000 and 0 <= bits <= 10");
  if (kind != RT_TABLE_CHORDS && kind != RT_TABLE_GREY_EXACT)
    return fail(RT_ERR_INVALID, "rt_set_tables: unknown table kind");
  const int S = K - 1;
  std::vector<double2> gc(S), hc(S);
  if (kind == RT_TABLE_CHORDS) {
    if (!h_g || !h_h) return fail(RT_ERR_INVALID, "rt_set_tables: knot arrays required");
    for (int k = 0; k < K; ++k)
      if (!std::isfinite(h_g[k]) || !std::isfinite(h_h[k]) || h_g[k] < 0 || h_h[k] < 0)
        return fail(RT_ERR_INVALID, "rt_set_tables: knot values must be finite and >= 0");
    auto tau = [&](int idx) {
      if (idx == 0) return 0.0;
      if (idx == K - 1) return std::ldexp(1.0, E1);
      const int t = idx - 1;
      return std::ldexp(1.0 + (double)(t & ((1 << bits) - 1)) / (double)(1 << bits), (t >> bits) - E0);
    };
    for (int s = 0; s < S; ++s) {
      const double tl = tau(s), th = tau(s + 1);
      double c1 = (h_g[s + 1] - h_g[s]) / (th - tl);
      gc[s] = make_double2(std::fma(-c1, tl, h_g[s]), c1);
      c1 = (h_h[s + 1] - h_h[s]) / (th - tl);
      hc[s] = make_double2(std::fma(-c1, tl, h_h[s]), c1);
    }
  }
  double2 *dg = nullptr, *dh = nullptr;
  TRY(dev_malloc(&dg, S * sizeof(double2)));
  cudaError_t e = dev_malloc(&dh, S * sizeof(double2));
  if (e == cudaSuccess) e = cudaMemcpy(dg, gc.data(), S * sizeof(double2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(dh, hc.data(), S * sizeof(double2), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    dev_free(dg);
    dev_free(dh);
    return cuda_fail(e, "rt_set_tables");
  }
  dev_free(g.gtab);
  dev_free(g.htab);
  g.gtab = dg;
  g.htab = dh;
  g.tab_kind = kind;
  g.E0 = E0;
  g.E1 = E1;
  g.B = bits;
  g.have_tables = true;
  ++g.epoch;
  return RT_OK;
}

static rt_status set_field(rt_grid_t h, const double* d, bool density) {
  const char* who = density ? "rt_set_density" : "rt_set_xHI";
  if (!h) return fail(RT_ERR_INVALID, std::string(who) + ": null grid");
  if (!d) return fail(RT_ERR_INVALID, std::string(who) + ": null field");
  Grid& g = *reinterpret_cast<Grid*>(h);
  int herr = 0;
  TRY(cudaMemsetAsync(g.err + 1, 0, sizeof(int), g.stream));
  TRY(launch_validate_fields(g, density ? d : nullptr, density ? nullptr : d));
  TRY(cudaMemcpyAsync(&herr, g.err + 1, sizeof(int), cudaMemcpyDeviceToHost, g.stream));
  TRY(cudaStreamSynchronize(g.stream));
  if (herr)
    return fail(RT_ERR_INVALID, density ? "rt_set_density: n_H must be finite, >= +0 and <= 1e12"
                                        : "rt_set_xHI: x_HI must lie in [+0, 1]");
  if (density) g.nH = d; else g.xHI = d;
  ++g.epoch;
  return RT_OK;
}

rt_status rt_set_scale_factor(rt_grid_t h, double a) {
  if (!h) return fail(RT_ERR_INVALID, "rt_set_scale_factor: null grid");
  if (!(a > 0.0) || !std::isfinite(a) || a > 1e6 || a < 1e-6)
    return fail(RT_ERR_INVALID, "rt_set_scale_factor: a must be finite and in [1e-6, 1e6]");
  Grid& g = *reinterpret_cast<Grid*>(h);
  g.a = a;
  g.inv_a3 = 1.0 / (a * a * a);
  for (int b = 0; b < g.nbox; ++b) set_box_cell(g.boxes_h[b], g.cell_comoving[b] * a, g.p.sigma0_cm2);
  TRY(cudaMemcpyAsync(g.boxes_d, g.boxes_h.data(), g.nbox * sizeof(BoxDev), cudaMemcpyHostToDevice,
                      g.stream));
  TRY(cudaStreamSynchronize(g.stream));  // the host records may change again
  ++g.epoch;
  return RT_OK;
}

rt_status rt_set_density(rt_grid_t h, const double* d_nH) { return set_field(h, d_nH, true); }
rt_status rt_set_xHI(rt_grid_t h, const double* d_xHI) { return set_field(h, d_xHI, false); }

rt_status rt_set_sources(rt_grid_t h, int nsrc, const int32_t* d_pos, const int32_t* d_box,
                         const double* d_ndot, const double* d_radius) {
  if (!h) return fail(RT_ERR_INVALID, "rt_set_sources: null grid");
  if (nsrc < 0 || nsrc > (1 << 26)) return fail(RT_ERR_INVALID, "rt_set_sources: bad source count");
  if (nsrc > 0 && (!d_pos || !d_ndot || !d_radius))
    return fail(RT_ERR_INVALID, "rt_set_sources: null source array");
  Grid& g = *reinterpret_cast<Grid*>(h);
  ++g.epoch;  // the source arrays, tables and geometry may move
  rt_status st = ingest_sources(g, nsrc, d_pos, d_box, d_ndot, d_radius);
  if (st == RT_OK) {
    const int mmax = std::max(1, std::min(isqrt_h(g.max_r2), g.nmax / 2 + 1));
    st = ensure_geometry(g, mmax);
  }
  if (st == RT_OK) st = ensure_row_tables(g);
  if (st != RT_OK) {  // no kernel may use sources whose geometry or tables are missing
    g.nsrc = 0;
    g.nsrc_in = 0;
    g.max_r2 = 0;
    g.source_voxels = 0;
    g.r2_sorted_h.clear();
  }
  return st;
}

rt_status rt_raytrace(rt_grid_t h, double* d_gamma, int schedule) {
  if (!h) return fail(RT_ERR_INVALID, "rt_raytrace: null grid");
  if (!d_gamma) return fail(RT_ERR_INVALID, "rt_raytrace: null output");
  if (schedule != RT_SCHED_AUTO && schedule != RT_SCHED_PLAIN && schedule != RT_SCHED_BATCHED &&
      schedule != RT_SCHED_BATCHED_EXIT)
    return fail(RT_ERR_INVALID, "rt_raytrace: unknown schedule");
  Grid& g = *reinterpret_cast<Grid*>(h);
  rt_status st = check_ready(g, "rt_raytrace");
  if (st != RT_OK) return st;
  TRY(cudaEventRecord(g.ev[0], g.stream));
  TRY(launch_precompute(g));
  TRY(cudaMemsetAsync(d_gamma, 0, g.ncell * sizeof(double), g.stream));
  TRY(cudaEventRecord(g.ev[1], g.stream));
  if (schedule == RT_SCHED_AUTO) schedule = g.auto_plain ? RT_SCHED_PLAIN : RT_SCHED_BATCHED;
  if (g.nsrc > 0) {
    if (schedule == RT_SCHED_PLAIN)
      st = run_trace(g, d_gamma, nullptr, nullptr, g.nsrc, RT_SCHED_PLAIN, g.nsrc);
    else
      st = run_trace(g, d_gamma, nullptr, g.items, 24 * g.nsrc, RT_SCHED_BATCHED, g.nsrc, nullptr,
                     schedule == RT_SCHED_BATCHED_EXIT);
    if (st != RT_OK) return st;
  } else {
    g.stats.launches = 0;
    g.stats.items = 0;
  }
  TRY(cudaEventRecord(g.ev[2], g.stream));
  g.stats.source_voxels = g.source_voxels;
  return RT_OK;
}

rt_status rt_raytrace_source_coldens(rt_grid_t h, int src, double* d_coldens, int schedule) {
  if (!h) return fail(RT_ERR_INVALID, "rt_raytrace_source_coldens: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  if (!d_coldens) return fail(RT_ERR_INVALID, "rt_raytrace_source_coldens: null output");
  if (src < 0 || src >= g.nsrc_in)
    return fail(RT_ERR_INVALID, "rt_raytrace_source_coldens: source index out of range");
  rt_status st = check_ready(g, "rt_raytrace_source_coldens");
  if (st != RT_OK) return st;
  int p = 0;
  TRY(cudaMemcpyAsync(&p, g.src_of_input + src, sizeof(int), cudaMemcpyDeviceToHost, g.stream));
  TRY(cudaStreamSynchronize(g.stream));
  int hitems[24];
  for (int q = 0; q < 24; ++q) hitems[q] = (p << 5) | q;
  TRY(cudaMemcpyAsync(g.queue + 8, hitems, 24 * sizeof(int), cudaMemcpyHostToDevice, g.stream));
  TRY(launch_precompute(g));
  TRY(cudaMemsetAsync(d_coldens, 0, g.ncell * sizeof(double), g.stream));
  if (schedule == RT_SCHED_PLAIN) {
    hitems[0] = p;
    TRY(cudaMemcpyAsync(g.queue + 8, hitems, sizeof(int), cudaMemcpyHostToDevice, g.stream));
    st = run_trace(g, nullptr, d_coldens, g.queue + 8, 1, RT_SCHED_PLAIN, 1);
  } else {
    st = run_trace(g, nullptr, d_coldens, g.queue + 8, 24, RT_SCHED_BATCHED, 0, nullptr, false,
                   g.r2_sorted_h[p]);
  }
  if (st != RT_OK) return st;
  TRY(cudaStreamSynchronize(g.stream));  // hitems is a stack buffer
  return latched_errors(g);
}

rt_status rt_get_stats(rt_grid_t h, rt_stats* out) {
  if (!h || !out) return fail(RT_ERR_INVALID, "rt_get_stats: null argument");
  Grid& g = *reinterpret_cast<Grid*>(h);
  TRY(cudaStreamSynchronize(g.stream));
  float ms = 0.f;
  if (cudaEventElapsedTime(&ms, g.ev[1], g.ev[2]) == cudaSuccess) g.stats.trace_ms = ms;
  if (cudaEventElapsedTime(&ms, g.ev[0], g.ev[1]) == cudaSuccess) g.stats.prep_ms = ms;
  cudaGetLastError();
  unsigned long long rc = 0;
  TRY(cudaMemcpy(&rc, g.counters, sizeof(rc), cudaMemcpyDeviceToHost));
  g.stats.rate_cells = (int64_t)rc;
  g.stats.kernel_launches = g_launches.load();
  g.stats.row_table_bytes = g.rtab ? g.rtab_bytes + g.itab_bytes : 0;
  *out = g.stats;
  return latched_errors(g);
}

rt_status rt_check(rt_grid_t h) {
  if (!h) return fail(RT_ERR_INVALID, "rt_check: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  TRY(cudaStreamSynchronize(g.stream));
  return latched_errors(g);
}

rt_status rt_inject_device_error(rt_grid_t h, int bits) {
  if (!h) return fail(RT_ERR_INVALID, "rt_inject_device_error: null grid");
  if (bits <= 0 || bits > (ERR_LAYER_CAP | ERR_GEO | ERR_INPUT | ERR_CUBE))
    return fail(RT_ERR_INVALID, "rt_inject_device_error: unknown error bits");
  Grid& g = *reinterpret_cast<Grid*>(h);
  int cur = 0;
  TRY(cudaStreamSynchronize(g.stream));
  TRY(cudaMemcpy(&cur, g.err, sizeof(int), cudaMemcpyDeviceToHost));
  cur |= bits;
  TRY(cudaMemcpy(g.err, &cur, sizeof(int), cudaMemcpyHostToDevice));
  return RT_OK;
}

rt_status rt_set_device_memory_limit(int64_t bytes) {
  if (bytes < 0) return fail(RT_ERR_INVALID, "rt_set_device_memory_limit: negative limit");
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  mem_limit_locked();  // the environment's value is replaced, not read later
  g_mem_limit = bytes;
  return RT_OK;
}

int64_t rt_device_memory_in_use(void) {
  std::lock_guard<std::mutex> lk(g_mem_mutex);
  return g_mem_live;
}

rt_status rt_chemistry_step(rt_grid_t h, const double* d_gamma, const double* d_x0,
                            const double* d_xavg_in, double dt_s, double alpha_H, double C_H,
                            double conv_tol, double* d_xavg_out, double* d_xnew_out,
                            int64_t* d_unconverged) {
  if (!h) return fail(RT_ERR_INVALID, "rt_chemistry_step: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  if (!d_gamma || !d_x0 || !d_xavg_in || !d_xavg_out || !d_xnew_out || !d_unconverged)
    return fail(RT_ERR_INVALID, "rt_chemistry_step: null pointer");
  if (!(dt_s > 0) || !std::isfinite(dt_s) || !(alpha_H >= 0) || !(C_H >= 0) || !(conv_tol >= 0))
    return fail(RT_ERR_INVALID, "rt_chemistry_step: need dt > 0, alpha_H >= 0, C_H >= 0");
  if (!g.nH) return fail(RT_ERR_STATE, "rt_chemistry_step: rt_set_density not called");
  TRY(launch_chemistry(g, d_gamma, d_x0, d_xavg_in, dt_s, alpha_H, C_H, 1e-10, 50, conv_tol,
                       d_xavg_out, d_xnew_out, d_unconverged, nullptr));
  return RT_OK;
}

rt_status rt_iterate(rt_grid_t h, double* d_x, double dt_s, double alpha_H, double C_H,
                     int max_iter, double conv_tol, double conv_frac, int use_graph,
                     double* d_gamma, int* h_iters) {
  if (!h) return fail(RT_ERR_INVALID, "rt_iterate: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  if (!d_x || !d_gamma) return fail(RT_ERR_INVALID, "rt_iterate: null pointer");
  if (max_iter < 1 || max_iter > 1000 || !(dt_s > 0) || !(alpha_H >= 0) || !(C_H >= 0) ||
      !(conv_tol >= 0) || !(conv_frac >= 0))
    return fail(RT_ERR_INVALID, "rt_iterate: bad arguments");
  if (!g.have_tables) return fail(RT_ERR_STATE, "rt_iterate: rt_set_tables not called");
  if (!g.nH) return fail(RT_ERR_STATE, "rt_iterate: rt_set_density not called");
  const size_t bytes = g.ncell * sizeof(double);
  if (!g.xbuf) {
    TRY(dev_malloc(&g.xbuf, bytes));
    TRY(dev_malloc(&g.xavg, bytes));
    TRY(dev_malloc(&g.xavg2, bytes));
    TRY(dev_malloc(&g.xhi_int, bytes));
  }
  g.xHI = g.xhi_int;
  const int64_t limit = (int64_t)std::ceil(conv_frac * (double)g.ncell);
  cudaStream_t user = g.stream;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  rt_status st = RT_OK;
  int iters = 0;
  auto body = [&](int k) -> rt_status {
    const int* skip = g.flags;
    double* xin = (k % 2 == 0) ? g.xavg : g.xavg2;
    double* xout = (k % 2 == 0) ? g.xavg2 : g.xavg;
    TRY(launch_one_minus(xin, g.xhi_int, g.ncell, skip, g.stream));
    TRY(launch_precompute(g, skip));
    TRY(launch_zero(d_gamma, g.ncell, skip, g.stream));
    TRY(cudaMemsetAsync(g.unconv, 0, sizeof(int64_t), g.stream));
    if (g.nsrc > 0) {
      rt_status s2 = run_trace(g, d_gamma, nullptr, g.items, 24 * g.nsrc, RT_SCHED_BATCHED, g.nsrc, skip);
      if (s2 != RT_OK) return s2;
    }
    TRY(launch_chemistry(g, d_gamma, d_x, xin, dt_s, alpha_H, C_H, 1e-10, 50, conv_tol, xout,
                         g.xbuf, g.unconv, skip));
    TRY(launch_conv_check(g.unconv, limit, g.flags, g.stream));
    return RT_OK;
  };
  TRY(cudaMemcpyAsync(g.xavg, d_x, bytes, cudaMemcpyDeviceToDevice, user));
  TRY(cudaMemsetAsync(g.flags, 0, 2 * sizeof(int), user));
  if (use_graph) {
    // capture once on a private stream; replay while the arguments and the grid's
    // state are those it was captured with
    const Grid::IterKey key{d_x, d_gamma, dt_s, alpha_H, C_H, conv_tol, conv_frac, max_iter,
                            g.epoch, user};
    if (!g.it_stream) TRY(cudaStreamCreateWithFlags(&g.it_stream, cudaStreamNonBlocking));
    cudaStream_t cap = g.it_stream;
    if (!g.it_exec || !(key == g.it_key)) {
      if (g.it_exec) {
        TRY(cudaStreamSynchronize(cap));  // the old graph may still run
        cudaGraphExecDestroy(g.it_exec);
        g.it_exec = nullptr;
      }
      g.stream = cap;
      g.capturing = true;
      cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        for (int k = 0; k < max_iter && st == RT_OK; ++k) st = body(k);
        cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
        if (st == RT_OK && e2 != cudaSuccess) st = cuda_fail(e2, "cudaStreamEndCapture");
      } else {
        st = cuda_fail(e, "cudaStreamBeginCapture");
      }
      g.capturing = false;
      g.stream = user;
      if (st == RT_OK) {
        cudaError_t e3 = cudaGraphInstantiate(&exec, graph, 0);
        if (e3 != cudaSuccess) st = cuda_fail(e3, "cudaGraphInstantiate");
      }
      if (graph) cudaGraphDestroy(graph);
      if (st != RT_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        return st;
      }
      g.it_exec = exec;
      g.it_key = key;
    }
    cudaError_t e4 = cudaEventRecord(g.ev[3], user);
    if (e4 == cudaSuccess) e4 = cudaStreamWaitEvent(cap, g.ev[3], 0);
    if (e4 == cudaSuccess) e4 = cudaGraphLaunch(g.it_exec, cap);
    if (e4 == cudaSuccess) e4 = cudaEventRecord(g.ev[3], cap);
    if (e4 == cudaSuccess) e4 = cudaStreamWaitEvent(user, g.ev[3], 0);
    if (e4 != cudaSuccess) return cuda_fail(e4, "graph launch");
  } else {
    for (int k = 0; k < max_iter; ++k) {
      st = body(k);
      if (st != RT_OK) return st;
      int fl[2] = {0, 0};
      TRY(cudaMemcpyAsync(fl, g.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, user));
      TRY(cudaStreamSynchronize(user));
      if (fl[0]) break;
    }
  }
  TRY(cudaMemcpyAsync(d_x, g.xbuf, bytes, cudaMemcpyDeviceToDevice, user));
  if (h_iters) {
    int fl[2] = {0, 0};
    TRY(cudaMemcpyAsync(fl, g.flags, 2 * sizeof(int), cudaMemcpyDeviceToHost, user));
    TRY(cudaStreamSynchronize(user));
    iters = fl[1];
    *h_iters = iters;
    return latched_errors(g);
  }
  return RT_OK;
}

rt_status rt_raytrace_backward(rt_grid_t h, const double* d_dL_dgamma, double* d_dL_dlog_nHI,
                               double* d_dL_dlog_ndot) {
  if (!h) return fail(RT_ERR_INVALID, "rt_raytrace_backward: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  if (!d_dL_dgamma || !d_dL_dlog_nHI)
    return fail(RT_ERR_INVALID, "rt_raytrace_backward: null pointer");
  if (g.nsrc_in > 0 && !d_dL_dlog_ndot)
    return fail(RT_ERR_INVALID, "rt_raytrace_backward: null dL/dlog Ndot output");
  rt_status st = check_ready(g, "rt_raytrace_backward");
  if (st != RT_OK) return st;
  if (g.interp_mode != RT_INTERP_GEOMETRIC)
    return fail(RT_ERR_INVALID, "rt_raytrace_backward: the adjoint is built for the geometric "
                                "weights (rt_set_interpolation mode 0)");
  TRY(launch_precompute(g));
  TRY(cudaMemsetAsync(d_dL_dlog_nHI, 0, g.ncell * sizeof(double), g.stream));
  if (g.nsrc == 0) return RT_OK;
  if (g.dq_cap < g.nsrc) {
    dev_free(g.dq_merged);
    g.dq_merged = nullptr;
    g.dq_cap = 0;
    TRY(dev_malloc(&g.dq_merged, g.nsrc * sizeof(double)));
    g.dq_cap = g.nsrc;
  }
  TRY(cudaMemsetAsync(g.dq_merged, 0, g.nsrc * sizeof(double), g.stream));
  // items of large sources by 128-thread CTAs, the rest one per warp (as the trace,
  // but with the warp-mode threshold capped at half-width 27: an adjoint warp keeps
  // two layers and its layer records in shared memory, and beyond 27 too few of
  // its warps stay resident -- 1e5 sources of the 250^3 workload took 1.5x longer
  // at 30)
  const int hbig = face_hcap(g.max_r2, g.nmax);
  const int lcap = std::max(1, std::min(isqrt_h(g.max_r2), g.nmax / 2 + 1));
  const int n_items = 24 * g.nsrc;
  const int hsmall_bwd = std::min(g.hsmall, 27);
  int split = n_items, hsm = 0, r2sm = 0;
  if (hsmall_bwd > 0 && !g.r2_sorted_h.empty()) {
    int lo = 0, hi = (int)g.r2_sorted_h.size();
    while (lo < hi) {
      const int mid = (lo + hi) / 2;
      if (face_hcap(g.r2_sorted_h[mid], g.nmax) <= hsmall_bwd) hi = mid; else lo = mid + 1;
    }
    if (lo < (int)g.r2_sorted_h.size()) {
      split = 24 * lo;
      hsm = face_hcap(g.r2_sorted_h[lo], g.nmax);
      r2sm = g.r2_sorted_h[lo];
    }
  }
  size_t smem_c = 0, smem_w = 0, cap_c = 0, cap_w = 0;
  int grid_c = 0, grid_w = 0;
  if (split > 0) {
    smem_c = bwd_smem_bytes(hbig, lcap);
    if (smem_c > 227 * 1024)
      return fail(RT_ERR_INVALID, "rt_raytrace_backward: radius too large for the shared-memory layers");
    cap_c = face_stack_cap(g.max_r2, g.nmax);
    const int maxg = bwd_max_grid(smem_c, 128);
    if (maxg <= 0) return fail(RT_ERR_CUDA, "rt_raytrace_backward: no occupancy");
    grid_c = std::max(1, std::min(split, maxg));
  }
  if (split < n_items) {
    smem_w = bwd_smem_bytes(hsm, lcap) * 8;
    cap_w = face_stack_cap(r2sm, g.nmax);
    const int maxg = bwd_max_grid(smem_w, 32);
    if (maxg <= 0) return fail(RT_ERR_CUDA, "rt_raytrace_backward: no occupancy (warp mode)");
    grid_w = std::max(1, std::min((n_items - split + 7) / 8, maxg));
  }
  const size_t need = (cap_c * (size_t)grid_c + cap_w * (size_t)grid_w * 8) * sizeof(double2);
  if (need > g.bwd_stack_bytes) {
    dev_free(g.bwd_stack);
    g.bwd_stack = nullptr;
    g.bwd_stack_bytes = 0;
    TRY(dev_malloc(&g.bwd_stack, need));
    g.bwd_stack_bytes = need;
  }
  TraceArgs a = base_args(g);
  a.items = g.items;
  TRY(cudaMemsetAsync(g.queue, 0, 2 * sizeof(int), g.stream));
  TRY(cudaEventRecord(g.ev[1], g.stream));
  g.stats.launches = 0;
  if (split > 0) {
    TraceArgs b = a;
    b.hcap = hbig;
    b.item_begin = 0;
    b.n_items = split;
    b.queue = g.queue;
    TRY(launch_trace_bwd(g, b, d_dL_dgamma, d_dL_dlog_nHI, g.dq_merged, g.bwd_stack, cap_c, lcap,
                         grid_c, smem_c, 128, g.bwd_exit != 0));
    g.stats.launches += 1;
  }
  if (split < n_items) {
    TraceArgs b = a;
    b.hcap = hsm;
    b.item_begin = split;
    b.n_items = n_items;
    b.queue = g.queue + 1;
    TRY(launch_trace_bwd(g, b, d_dL_dgamma, d_dL_dlog_nHI, g.dq_merged,
                         g.bwd_stack + cap_c * (size_t)grid_c, cap_w, lcap, grid_w, smem_w, 32,
                         g.bwd_exit != 0));
    g.stats.launches += 1;
  }
  TRY(cudaEventRecord(g.ev[2], g.stream));
  TRY(launch_dndot_inputs(g, g.dq_merged, d_dL_dlog_ndot));
  g.stats.block = split > 0 ? 128 : 32;
  g.stats.grid = split > 0 ? grid_c : grid_w;
  g.stats.items = n_items;
  return RT_OK;
}

rt_status rt_set_interpolation(rt_grid_t h, int mode, double tau_weight_min) {
  if (!h) return fail(RT_ERR_INVALID, "rt_set_interpolation: null grid");
  if (mode != RT_INTERP_GEOMETRIC && mode != RT_INTERP_OPTICAL_DEPTH)
    return fail(RT_ERR_INVALID, "rt_set_interpolation: unknown mode");
  if (!(tau_weight_min > 0.0) || !std::isfinite(tau_weight_min))
    return fail(RT_ERR_INVALID, "rt_set_interpolation: tau_weight_min must be finite and > 0");
  Grid& g = *reinterpret_cast<Grid*>(h);
  g.interp_mode = mode;
  g.tau_w0 = tau_weight_min;
  ++g.epoch;
  return RT_OK;
}

rt_status rt_set_adjoint_mode(rt_grid_t h, int stop_at_opaque) {
  if (!h) return fail(RT_ERR_INVALID, "rt_set_adjoint_mode: null grid");
  reinterpret_cast<Grid*>(h)->bwd_exit = stop_at_opaque ? 1 : 0;
  return RT_OK;
}

rt_status rt_set_schedule(rt_grid_t h, int block_big, int hsmall, int hface) {
  if (!h) return fail(RT_ERR_INVALID, "rt_set_schedule: null grid");
  if (block_big != 128 && block_big != 256)
    return fail(RT_ERR_INVALID, "rt_set_schedule: block must be 128 or 256");
  if (hsmall < 0 || hsmall > 32)
    return fail(RT_ERR_INVALID, "rt_set_schedule: hsmall must be 0..32");
  if (hface < 0 || hface > 20)
    return fail(RT_ERR_INVALID, "rt_set_schedule: hface must be 0..20");
  Grid& g = *reinterpret_cast<Grid*>(h);
  g.block_big = block_big;
  g.hsmall = hsmall;
  g.hface = hface;
  ++g.epoch;
  return RT_OK;
}

// Key of a workload for the autotuner cache: box sizes and the distribution of
// traced radii (what the schedule's performance depends on).
static std::string tune_key(const Grid& g) {
  std::vector<int> r2 = g.r2_sorted_h;  // descending
  auto pct = [&](double q) { return r2.empty() ? 0 : r2[(size_t)((1.0 - q) * (r2.size() - 1))]; };
  std::ostringstream k;
  k << "nbox=" << g.nbox << ",nmax=" << g.nmax << ",ncell=" << g.ncell << ",nsrc=" << g.nsrc
    << ",r2max=" << g.max_r2 << ",r2p50=" << pct(0.5) << ",r2p90=" << pct(0.9);
  return k.str();
}

rt_status rt_autotune(rt_grid_t h, const char* cache_path, int* h_block, int* h_hsmall,
                      int* h_hface) {
  if (!h) return fail(RT_ERR_INVALID, "rt_autotune: null grid");
  Grid& g = *reinterpret_cast<Grid*>(h);
  ++g.epoch;  // the schedule may change
  rt_status st = check_ready(g, "rt_autotune");
  if (st != RT_OK) return st;
  auto report = [&]() {
    if (h_block) *h_block = g.block_big;
    if (h_hsmall) *h_hsmall = g.hsmall;
    if (h_hface) *h_hface = g.hface;
  };
  const std::string key = tune_key(g);
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      std::istringstream ls(line);
      std::string k;
      int b = 0, hs = -1, hf = -1, ap = -1;
      if ((ls >> k >> b >> hs >> hf >> ap) && k == key && (b == 128 || b == 256) && hs >= 0 &&
          hs <= 32 && hf >= 0 && hf <= 20 && (ap == 0 || ap == 1)) {
        g.block_big = b;
        g.hsmall = hs;
        g.hface = hf;
        g.auto_plain = ap;
        report();
        return RT_OK;
      }
    }
  }
  if (g.nsrc == 0) {
    report();
    return RT_OK;
  }
  double* gam = nullptr;
  TRY(dev_malloc(&gam, g.ncell * sizeof(double)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // time of one batched trace in the current configuration (second of two runs)
  auto timed = [&](float& t) {
    for (int rep = 0; rep < 2 && st == RT_OK; ++rep) {
      cudaEventRecord(e0, g.stream);
      st = rt_raytrace(h, gam, RT_SCHED_BATCHED);
      cudaEventRecord(e1, g.stream);
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&t, e0, e1);
    }
    return st == RT_OK;
  };
  // stage 1: CTA size x warp-mode threshold (whole-face warps off); stage 2: the
  // whole-face threshold at the chosen pair
  const int blocks[] = {128, 256};
  const int hss[] = {0, 11, 15, 19, 22, 24, 27, 30};
  const int hfs[] = {9, 11, 13, 15, 17, 19};
  float best = 1e30f;
  int bb = g.block_big, bh = g.hsmall, bf = 0;
  g.hface = 0;
  for (int b : blocks)
    for (int hs : hss) {
      if (st != RT_OK) break;
      g.block_big = b;
      g.hsmall = hs;
      float t = 0.f;
      if (!timed(t)) break;
      if (t < best) {
        best = t;
        bb = b;
        bh = hs;
      }
    }
  g.block_big = bb;
  g.hsmall = bh;
  for (int hf : hfs) {
    if (st != RT_OK || bh == 0) break;
    g.hface = hf;
    float t = 0.f;
    if (!timed(t)) break;
    if (t < best) {
      best = t;
      bf = hf;
    }
  }
  // stage 2b: the warp-mode threshold again, with the chosen whole-face threshold
  // (whole faces take the small sources away from the warp mode, which shifts its
  // best range)
  if (bf > 0) {
    g.hface = bf;
    for (int hs : hss) {
      if (st != RT_OK) break;
      if (hs == 0 || hs == bh) continue;
      g.hsmall = hs;
      float t = 0.f;
      if (!timed(t)) break;
      if (t < best) {
        best = t;
        bh = hs;
      }
    }
    g.hsmall = bh;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  dev_free(gam);
  if (st != RT_OK) return st;
  g.hface = bf;
  // stage 3: the paper's block-per-source schedule against the tuned batched one
  // (RT_SCHED_AUTO then takes the faster)
  if (st == RT_OK) {
    float tp = 0.f;
    TRY(dev_malloc(&gam, g.ncell * sizeof(double)));
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, g.stream);
    st = rt_raytrace(h, gam, RT_SCHED_PLAIN);
    cudaEventRecord(e1, g.stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(&tp, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dev_free(gam);
    if (st != RT_OK) return st;
    g.auto_plain = tp < best ? 1 : 0;
  }
  report();
  if (cache_path) {
    std::ofstream out(cache_path, std::ios::app);
    out << key << " " << bb << " " << bh << " " << bf << " " << g.auto_plain << "\n";
  }
  return RT_OK;
}

void rt_grid_destroy(rt_grid_t h) {
  if (!h) return;
  Grid* g = reinterpret_cast<Grid*>(h);
  cudaStreamSynchronize(g->stream);
  free_grid(g);
}

}  // extern "C"
