// Internal declarations shared by the CUDA translation units of libasora.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <map>
#include <vector>

#include "../../include/asora.h"

namespace asora {

// ------------------------------------------------------------------ boxes
struct BoxDev {
  int n;            // cells per side
  int wlo, whi;     // periodic window of offsets: [-n/2, n/2-1] (even), [-(n-1)/2,(n-1)/2] (odd)
  int64_t off;      // first cell of this box in the concatenated fields
  double cell;      // cell size (cm)
  double inv_cell3; // 1/cell^3
  double thin_fac;  // sigma0 / cell^2
  double sig_cell;  // sigma0 * cell
};

// Source after ingest (merged, LPT ordered).
struct SrcDev {
  int i, j, k, box;
};

// Geometry of one canonical offset (m = |Delta_d| dominant, lo <= hi the two
// transverse magnitudes), source- and box-independent:
//   x = lo/m, y = hi/m,  W1 = (1-x)(1-y), WA = x(1-y), WB = (1-x)y, W4 = xy,
//   ds = sqrt(1 + (lo^2+hi^2)/m^2), invV = 1/(4 pi r2 ds), thin = 1/(4 pi r2),
//   r2 = m^2 + lo^2 + hi^2 (cells^2).
struct __align__(16) GeoEntry {
  double w1, wa, wb, w4;
  double ds, invv, thin, pad;
};
// Index of (m, lo, hi), 1 <= m, 0 <= lo <= hi <= m.
__host__ __device__ inline int64_t geo_index(int m, int lo, int hi) {
  return (int64_t)(m + 2) * (m + 1) * m / 6 - 1 + (int64_t)hi * (hi + 1) / 2 + lo;
}
inline int64_t geo_count(int mmax) { return geo_index(mmax + 1, 0, 0); }

// Row-major geometry for the batched trace: entry (m, a1, a2), 0 <= a1, a2 <= m,
// holds the weights in the cell's own orientation (a = a1/m, b = a2/m):
//   w1 = (1-a)(1-b), w2 = a(1-b), w3 = (1-a)b, w4 = ab, ds = sqrt(1 + (a1^2+a2^2)/m^2)
// (bit-identical to the (lo, hi) table's values; consecutive a2 are adjacent).
struct __align__(16) GeoRow {
  double w1, w2, w3, w4;
  double ds, pad;
};
__host__ __device__ inline int64_t georow_index(int m, int a1, int a2) {
  return (int64_t)m * (m + 1) * (2 * m + 1) / 6 - 1 + (int64_t)a1 * (m + 1) + a2;
}
inline int64_t georow_count(int mmax) { return georow_index(mmax + 1, 0, 0); }

// Rate tables on the device.
struct TabDev {
  const double2* g;  // (c0, c1) per segment
  const double2* h;
  int kind;          // RT_TABLE_*
  int E0, B;
  uint64_t tau_min_bits, tau_max_bits;  // bits of 2^-E0 and of the "no transmission" bound
};

// Arguments of the trace kernels.
struct TraceArgs {
  const BoxDev* boxes;
  const double* dtau;    // sigma0*cell*n_H*x_HI, C order per box
  const double* dtauT;   // the same, axes rotated to (k, i, j) per box
  const double* invn;    // 1/(n_H x_HI)
  double* gamma;         // output rates (may be null)
  double* coldens;       // optional per-source column density output
  const SrcDev* src;
  const double* ndot;
  const int* r2lim;      // floor(R^2) per source
  const int* items;      // (source << 5) | (face << 2) | quadrant, LPT order
  int item_begin;        // first item of this launch (the queue counts from here)
  int n_items;           // one past the last item of this launch
  int* queue;            // work counter
  const GeoEntry* geo;
  const GeoRow* georow;
  int geo_mmax;
  TabDev tab;
  double tau_lim;
  double sigma0;
  int hcap;              // layer half-size capacity (faces) / cube half-size (shells)
  double* scratch;       // per-CTA scratch (shell kernel)
  int* err;              // error flag (bit mask)
  const int* skip;       // if non-null and *skip != 0 the launch does nothing
  unsigned long long* rate_cells;  // number of rate evaluations (may be null)
  int early_exit;        // stop an item once a whole layer is opaque (rates only)
  double neg_zero;       // -0.0 at run time: fma(x, y, -0.0) is x*y bit for bit, as a DFMA
  int interp_mode;       // 0: geometric weights (Eq. interp); 1: optical-depth-modulated
  double tau_w0;         // floor of the modulation 1/max(tau_n, tau_w0) (mode 1)
  uint64_t exit_bits;    // bits of the opacity bound 2^E1 (1 + 2^-40)
  // Row tables of unclipped quadrant layers, one blob per (R^2 limit, m):
  // first flat index of rows 0..H+1 (ints) then the row of every flat index
  // (bytes), padded to 16 bytes.  Blob of layer m of an item with limit r2:
  // rtab + rtab_off[rtab_first[rtab_slot[r2]] + m - 1] (rtab_slot[r2] < 0: none).
  const unsigned char* rtab;
  const int* rtab_off;    // byte offset of every blob, plus one past the last
  const int* rtab_first;  // first blob of each R^2 limit
  const int* rtab_hcap;   // largest layer half-width of each R^2 limit
  const int* rtab_slot;   // R^2 limit -> slot, for 0..rtab_max_r2
  int rtab_max_r2;        // -1: no tables
  // Interior row tables of the same (R^2 limit, m) layers, for faces traced
  // whole (see k_interior_tables): blob of layer m at itab + itab_off[same index].
  const unsigned char* itab;
  const int* itab_off;
};

enum ErrBits { ERR_LAYER_CAP = 1, ERR_GEO = 2, ERR_INPUT = 4, ERR_CUBE = 8 };

// ----------------------------------------------------------- grid (handle)
struct Grid {
  int nbox = 0;
  std::vector<BoxDev> boxes_h;
  BoxDev* boxes_d = nullptr;
  int64_t ncell = 0;
  int nmax = 0;
  rt_params p{};
  cudaStream_t stream = nullptr;

  // tables
  bool have_tables = false;
  int tab_kind = 0, E0 = 0, E1 = 0, B = 0;
  double2* gtab = nullptr;
  double2* htab = nullptr;

  // expanding background: proper cell = comoving cell * a, proper n_H = n_H * inv_a3
  double a = 1.0;
  double inv_a3 = 1.0;
  std::vector<double> cell_comoving;  // per box, as created

  // inputs (borrowed)
  const double* nH = nullptr;
  const double* xHI = nullptr;
  bool dirty_fields = true;

  // derived per-cell fields (owned)
  double* dtau = nullptr;
  double* dtauT = nullptr;
  double* invn = nullptr;

  // sources (owned, ingested)
  int nsrc_in = 0;         // as given
  int nsrc = 0;            // after merging
  SrcDev* src = nullptr;
  double* ndot = nullptr;
  int* r2lim = nullptr;
  int* items = nullptr;    // 24 (face, quadrant) per source, LPT order
  int* src_of_input = nullptr;  // merged index of each input source
  double* ndot_in = nullptr;    // input photon rates (for the adjoint of merged sources)
  int max_r2 = 0;
  int64_t source_voxels = 0;
  std::vector<int> r2_sorted_h;  // per merged source (LPT order), host copy
  size_t src_cap = 0;            // sources the arrays above (and items / 24) can hold
  std::map<std::pair<int, int>, int64_t> ball_memo;  // traced cells per (R^2 limit, box size)
  // scratch of the source ingest, kept between calls and grown on demand
  struct Ingest {
    size_t cap = 0;  // sources the per-source arrays hold
    uint64_t *keys = nullptr, *keys2 = nullptr;
    int *idx = nullptr, *idx2 = nullptr, *r2in = nullptr, *head = nullptr, *mid = nullptr;
    SrcDev* msrc = nullptr;
    double* mndot = nullptr;
    int* mr2 = nullptr;
    uint32_t *lkey = nullptr, *lkey2 = nullptr;
    int *lval = nullptr, *order = nullptr, *lpt = nullptr;
    void* tmp = nullptr;
    size_t tmp_bytes = 0;
    int* dscal = nullptr;      // device scalars: [0] largest r2
    int* hscal = nullptr;      // pinned host: error bits, last head, last offset, largest r2
    int* r2pin = nullptr;      // pinned host: r2 per merged source
    SrcDev* srcpin = nullptr;  // pinned host: merged sources (ensembles)
  } ing;

  // precomputed row tables of the batched trace (see TraceArgs::rtab)
  unsigned char* rtab = nullptr;
  int* rtab_off = nullptr;
  int* rtab_first = nullptr;
  int* rtab_hcap = nullptr;
  int* rtab_slot = nullptr;
  int rtab_max_r2 = -1;
  int rtab_mcap = 0;
  int64_t rtab_bytes = 0;
  unsigned char* itab = nullptr;  // interior row tables (faces traced whole)
  int* itab_off = nullptr;
  int64_t itab_bytes = 0;
  std::vector<int> rtab_r2s;  // the R^2 limits the tables were built for (descending)

  // geometry
  GeoEntry* geo = nullptr;
  GeoRow* georow = nullptr;
  int geo_mmax = 0;

  // scratch
  int* queue = nullptr;
  int* err = nullptr;
  double* cube = nullptr;       // shell-kernel scratch
  size_t cube_bytes = 0;
  int64_t* unconv = nullptr;    // iteration counters
  double* xbuf = nullptr;       // rt_iterate buffers
  double* xavg = nullptr;
  double* xavg2 = nullptr;
  double* xhi_int = nullptr;
  int* flags = nullptr;
  int block_big = 128;      // threads per CTA for large-source items
  int hsmall = 19;          // items whose layers fit this half-width run one per warp
  int hface = 13;           // ... and those fitting this one whole faces per warp
  int auto_plain = 0;       // RT_SCHED_AUTO takes the plain schedule (autotuner's choice)
  int warps_per_block = 8;  // warp-mode CTA size of the last trace (1..8 warps)
  unsigned long long* counters = nullptr;  // [0]: rate evaluations of the last trace
  double2* bwd_stack = nullptr;  // adjoint: per-CTA (tau_in, tau_out) stacks
  size_t bwd_stack_bytes = 0;
  double* dq_merged = nullptr;   // adjoint: dL/dlog Ndot per merged source
  int dq_cap = 0;
  int bwd_exit = 1;              // adjoint: stop each item's recompute at its first opaque layer
  int interp_mode = 0;           // interpolation weights (rt_set_interpolation)
  double tau_w0 = 0.6;
  bool capturing = false;
  // rt_iterate's CUDA graph, kept for the next call with the same arguments and
  // no state change in between (epoch: bumped by every call that changes a
  // pointer, a launch configuration or a value a captured kernel uses)
  uint64_t epoch = 0;
  cudaGraphExec_t it_exec = nullptr;
  cudaStream_t it_stream = nullptr;
  struct IterKey {
    double* x = nullptr;
    double* gamma = nullptr;
    double dt = 0, alpha = 0, C = 0, conv_tol = 0, conv_frac = 0;
    int max_iter = 0;
    uint64_t epoch = 0;
    cudaStream_t user = nullptr;
    bool operator==(const IterKey& o) const {
      return x == o.x && gamma == o.gamma && dt == o.dt && alpha == o.alpha && C == o.C &&
             conv_tol == o.conv_tol && conv_frac == o.conv_frac && max_iter == o.max_iter &&
             epoch == o.epoch && user == o.user;
    }
  } it_key;

  // stats
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  rt_stats stats{};
};

// Kernels launched by this library in this process (host-side count).
void count_launch(int n = 1);

// Device allocations of the library: cudaMalloc/cudaFree with a process-wide
// cap on the bytes held (rt_set_device_memory_limit, or the environment
// variable ASORA_DEVICE_MEMORY_LIMIT); an allocation beyond the cap fails with
// cudaErrorMemoryAllocation (RT_ERR_OOM) without calling cudaMalloc.
cudaError_t dev_malloc_raw(void** p, size_t bytes);
cudaError_t dev_free(void* p);
template <class T>
inline cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc_raw(reinterpret_cast<void**>(p), bytes);
}

// Frees the source arrays and the ingest scratch (prep.cu).
void free_sources(Grid& g);

// Row tables for the distinct R^2 limits of the ingested sources (prep.cu);
// kept while the set of limits and the window size do not change.
rt_status ensure_row_tables(Grid& g);
void free_row_tables(Grid& g);

// error reporting (api.cu)
rt_status fail(rt_status st, const std::string& msg);
rt_status cuda_fail(cudaError_t e, const char* what);

// launchers (defined in the kernel translation units)
cudaError_t launch_precompute(Grid& g, const int* skip = nullptr);
cudaError_t launch_zero(double* p, int64_t n, const int* skip, cudaStream_t s);
cudaError_t launch_validate_fields(Grid& g, const double* nH, const double* xHI);
cudaError_t launch_geometry(GeoEntry* geo, GeoRow* georow, int mmax, cudaStream_t s);
cudaError_t launch_trace_faces(Grid& g, const TraceArgs& a, int block, int grid, size_t smem,
                               int wpb = 8);  // wpb: warps per CTA in warp mode (block 32)
cudaError_t launch_trace_shells(Grid& g, const TraceArgs& a, int block, int grid);
// per CTA (block 32, 4: per warp); od: with the reciprocal buffers of mode 1
size_t faces_smem_bytes(int hcap, int block, bool od = false);
int faces_max_grid(int block, size_t smem, int wpb = 8, bool od = false);
int shells_max_grid(int block);
rt_status ingest_sources(Grid& g, int nsrc, const int32_t* d_pos, const int32_t* d_box,
                         const double* d_ndot, const double* d_radius);
cudaError_t launch_chemistry(Grid& g, const double* gamma, const double* x0, const double* xavg_in,
                             double dt, double alpha_H, double C_H, double tol, int maxit,
                             double conv_tol, double* xavg_out, double* xnew_out,
                             int64_t* unconv, const int* skip_flag);
cudaError_t launch_one_minus(const double* x, double* y, int64_t n, const int* skip_flag,
                             cudaStream_t s);
size_t face_stack_cap(int r2, int nmax);
size_t bwd_smem_bytes(int hcap, int lcap);
int bwd_max_grid(size_t smem, int block);
cudaError_t launch_trace_bwd(Grid& g, const TraceArgs& t, const double* w, double* dlogn,
                             double* dndot_merged, double2* stack, size_t stack_cap, int lcap,
                             int grid, size_t smem, int block, bool exit);
cudaError_t launch_dndot_inputs(Grid& g, const double* dmerged, double* out);
cudaError_t launch_conv_check(const int64_t* unconv, int64_t limit, int* flag, cudaStream_t s);

}  // namespace asora
