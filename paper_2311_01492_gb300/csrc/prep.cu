// Per-call preparation kernels: field validation, per-cell optical depth
// (Sec. 3.1: dtau = sigma0 * alpha * n_HI), its axis-rotated copy for the
// z faces, 1/n_HI, the source-independent geometry table and source ingest
// (merging of co-located sources, Sec. 3, and longest-first ordering).
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <map>

#include "asora_internal.cuh"

namespace asora {

// ----------------------------------------------------------- validation
// (writes its own error word, g.err[1], so that it never clears the bits the
// trace kernels latch in g.err[0])
__global__ void k_validate_fields(const BoxDev* __restrict__ boxes, int nbox,
                                  const double* __restrict__ nH, const double* __restrict__ xHI,
                                  int64_t ncell, int* __restrict__ err) {
  int bad = 0;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    if (nH) {
      const double v = nH[c];
      if (!(v >= 0.0) || !isfinite(v) || signbit(v) || v > 1e12) bad = 1;
    }
    if (xHI) {
      const double v = xHI[c];
      if (!(v >= 0.0) || !(v <= 1.0) || signbit(v)) bad = 1;
    }
  }
  if (bad) atomicOr(err, ERR_INPUT);
}

cudaError_t launch_validate_fields(Grid& g, const double* nH, const double* xHI) {
  k_validate_fields<<<1024, 256, 0, g.stream>>>(g.boxes_d, g.nbox, nH, xHI, g.ncell, g.err + 1);
  count_launch();
  return cudaGetLastError();
}

// --------------------------------------------------------- per-cell fields
// One 32x32 tile of the (n^2 rows (i,j)) x (n cols k) matrix of a box:
// dtau = ((sigma0*cell)*n_H)*x_HI, invn = 1/(n_H*x_HI), and the transposed
// copy dtauT[k][i][j] so that the z faces read rows of constant k contiguously.
// n_H is the proper density: the given (comoving) one times inv_a3 = a^-3 in an
// expanding background (inv_a3 = 1 otherwise, an exact no-op); cell (in the
// box records) is the proper cell size.
__global__ void k_precompute(const BoxDev* __restrict__ boxes, const double* __restrict__ nH,
                             const double* __restrict__ xHI, double inv_a3,
                             double* __restrict__ dtau, double* __restrict__ dtauT,
                             double* __restrict__ invn, const int* __restrict__ skip) {
  __shared__ double tile[32][33];
  if (skip && *skip) return;
  const BoxDev B = boxes[blockIdx.z];
  const int n = B.n;
  const int64_t rows = (int64_t)n * n;
  const int c0 = blockIdx.x * 32;
  if (c0 >= n) return;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int64_t r0 = (int64_t)blockIdx.y * 32; r0 < rows; r0 += (int64_t)gridDim.y * 32) {
    for (int yy = ty; yy < 32; yy += 8) {
      const int64_t r = r0 + yy;
      const int c = c0 + tx;
      if (r < rows && c < n) {
        const int64_t idx = B.off + r * n + c;
        const double nh = nH[idx] * inv_a3, x = xHI[idx];
        const double d = (B.sig_cell * nh) * x;
        dtau[idx] = d;
        invn[idx] = 1.0 / (nh * x);
        tile[yy][tx] = d;
      }
    }
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
      const int c = c0 + yy;        // k
      const int64_t r = r0 + tx;    // (i,j)
      if (r < rows && c < n) dtauT[B.off + (int64_t)c * rows + r] = tile[tx][yy];
    }
    __syncthreads();
  }
}

cudaError_t launch_precompute(Grid& g, const int* skip) {
  const int n = g.nmax;
  dim3 grid((n + 31) / 32, (unsigned)std::min<int64_t>(((int64_t)n * n + 31) / 32, 65535), g.nbox);
  k_precompute<<<grid, dim3(32, 8), 0, g.stream>>>(g.boxes_d, g.nH, g.xHI, g.inv_a3, g.dtau,
                                                    g.dtauT, g.invn, skip);
  count_launch();
  return cudaGetLastError();
}

__global__ void k_zero(double* __restrict__ p, int64_t n, const int* __restrict__ skip) {
  if (skip && *skip) return;
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    p[c] = 0.0;
}

cudaError_t launch_zero(double* p, int64_t n, const int* skip, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 8);
  k_zero<<<grid, 256, 0, s>>>(p, n, skip);
  count_launch();
  return cudaGetLastError();
}

// ------------------------------------------------------------- geometry
// Entry (m, lo, hi): bilinear weights of Sec. 3.1 for a = lo/m, b = hi/m and
// the path length ds = sqrt(1 + (lo^2+hi^2)/m^2).  Both are computed with
// correctly rounded IEEE division and square root.
__global__ void k_geometry(GeoEntry* __restrict__ geo, int mmax) {
  const int m = blockIdx.x + 1;
  if (m > mmax) return;
  const int cnt = (m + 1) * (m + 2) / 2;
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    int hi = (int)((sqrtf(8.0f * t + 1.0f) - 1.0f) * 0.5f);
    while (hi * (hi + 1) / 2 > t) --hi;
    while ((hi + 1) * (hi + 2) / 2 <= t) ++hi;
    const int lo = t - hi * (hi + 1) / 2;
    const double x = (double)lo / (double)m;
    const double y = (double)hi / (double)m;
    GeoEntry e;
    e.w1 = (1.0 - x) * (1.0 - y);
    e.wa = x * (1.0 - y);
    e.wb = (1.0 - x) * y;
    e.w4 = x * y;
    e.ds = sqrt(1.0 + (double)(lo * lo + hi * hi) / (double)(m * m));
    const double r2 = (double)(m * m + lo * lo + hi * hi);
    const double fourpi = 12.566370614359172;
    e.invv = 1.0 / (fourpi * r2 * e.ds);
    e.thin = 1.0 / (fourpi * r2);
    e.pad = 0.0;
    geo[geo_index(m, lo, hi)] = e;
  }
}

// Row-major entry (m, a1, a2) with the same correctly rounded expressions.
__global__ void k_geometry_rows(GeoRow* __restrict__ geo, int mmax) {
  const int m = blockIdx.x + 1;
  if (m > mmax) return;
  const int cnt = (m + 1) * (m + 1);
  for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
    const int a1 = t / (m + 1), a2 = t - a1 * (m + 1);
    const double x = (double)a1 / (double)m;
    const double y = (double)a2 / (double)m;
    GeoRow e;
    e.w1 = (1.0 - x) * (1.0 - y);
    e.w2 = x * (1.0 - y);
    e.w3 = (1.0 - x) * y;
    e.w4 = x * y;
    e.ds = sqrt(1.0 + (double)(a1 * a1 + a2 * a2) / (double)(m * m));
    e.pad = 0.0;
    geo[georow_index(m, a1, a2)] = e;
  }
}

cudaError_t launch_geometry(GeoEntry* geo, GeoRow* georow, int mmax, cudaStream_t s) {
  if (mmax < 1) return cudaSuccess;
  k_geometry_rows<<<mmax, 256, 0, s>>>(georow, mmax);
  count_launch();
  k_geometry<<<mmax, 256, 0, s>>>(geo, mmax);
  count_launch();
  return cudaGetLastError();
}

// --------------------------------------------------------- source ingest
__global__ void k_src_keys(const BoxDev* __restrict__ boxes, int nbox, int nsrc,
                           const int32_t* __restrict__ pos, const int32_t* __restrict__ box,
                           const double* __restrict__ ndot, const double* __restrict__ radius,
                           uint64_t* __restrict__ keys, int* __restrict__ idx,
                           int* __restrict__ r2out, int* __restrict__ err) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nsrc) return;
  const int b = box ? box[s] : 0;
  bool bad = b < 0 || b >= nbox;
  const BoxDev B = boxes[bad ? 0 : b];
  const int i = pos[3 * s], j = pos[3 * s + 1], k = pos[3 * s + 2];
  bad |= i < 0 || i >= B.n || j < 0 || j >= B.n || k < 0 || k >= B.n;
  const double R = radius[s], nd = ndot[s];
  bad |= !(R > 0.0) || !isfinite(R) || !(nd >= 0.0) || !isfinite(nd) || signbit(nd);
  // traced cells satisfy |Delta|^2 <= floor(R^2); every window cell has
  // |Delta|^2 <= 3 (n/2)^2, so larger limits trace the same set.
  const double cap = 3.0 * (double)(B.n / 2) * (double)(B.n / 2) + 1.0;
  const double rr = fmin(floor(R * R), cap);
  const int r2 = bad ? 0 : (int)rr;
  if (bad) atomicOr(err, ERR_INPUT);
  const int64_t cell = bad ? 0 : B.off + ((int64_t)i * B.n + j) * B.n + k;
  keys[s] = ((uint64_t)cell << 22) | (uint64_t)r2;
  idx[s] = s;
  r2out[s] = r2;
}

__global__ void k_src_heads(const uint64_t* __restrict__ keys, int nsrc, int* __restrict__ head) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsrc) return;
  head[t] = (t == 0 || keys[t] != keys[t - 1]) ? 1 : 0;
}

// Merged source m = segment starting at sorted position t: rates summed in
// input order; LPT sort key = (max_r2 - r2) ascending.
__global__ void k_src_merge(const uint64_t* __restrict__ keys, const int* __restrict__ idx,
                            const int* __restrict__ head, const int* __restrict__ mid, int nsrc,
                            const int32_t* __restrict__ pos, const int32_t* __restrict__ box,
                            const double* __restrict__ ndot, const int* __restrict__ r2in,
                            SrcDev* __restrict__ msrc, double* __restrict__ mndot,
                            int* __restrict__ mr2, uint32_t* __restrict__ lkey,
                            int* __restrict__ lval, int* __restrict__ src_of_input, int max_r2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nsrc) return;
  // mid = exclusive scan of head flags: a segment head's own index; any other
  // member sees its head counted already.
  const int m = mid[t] + head[t] - 1;
  src_of_input[idx[t]] = m;  // merged index, remapped to LPT order later
  if (!head[t]) return;
  const int s0 = idx[t];
  double sum = 0.0;
  for (int u = t; u < nsrc && (u == t || !head[u]); ++u) sum += ndot[idx[u]];
  SrcDev d;
  d.i = pos[3 * s0];
  d.j = pos[3 * s0 + 1];
  d.k = pos[3 * s0 + 2];
  d.box = box ? box[s0] : 0;
  msrc[m] = d;
  mndot[m] = sum;
  mr2[m] = r2in[s0];
  lkey[m] = (uint32_t)(max_r2 - r2in[s0]);
  lval[m] = m;
}

// Permute merged sources into LPT order and emit 24 (face, quadrant) items per source.
__global__ void k_src_order(const int* __restrict__ order, int nm, const SrcDev* __restrict__ msrc,
                            const double* __restrict__ mndot, const int* __restrict__ mr2,
                            SrcDev* __restrict__ src, double* __restrict__ ndot,
                            int* __restrict__ r2lim, int* __restrict__ items,
                            int* __restrict__ lpt_of_merged) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nm) return;
  const int m = order[p];
  src[p] = msrc[m];
  ndot[p] = mndot[m];
  r2lim[p] = mr2[m];
  lpt_of_merged[m] = p;
  for (int q = 0; q < 24; ++q) items[24 * p + q] = (p << 5) | q;  // face = q >> 2, quadrant = q & 3
}

__global__ void k_remap(int* __restrict__ a, const int* __restrict__ map, int n) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) a[t] = map[a[t]];
}

static int64_t ball_count(int r2, int n) {
  const int wlo = -(n / 2), whi = (n % 2 == 0) ? n / 2 - 1 : n / 2;
  int64_t cnt = 0;
  const int L = std::min((int)std::floor(std::sqrt((double)r2)) + 1, n);
  for (int a = std::max(-L, wlo); a <= std::min(L, whi); ++a)
    for (int b = std::max(-L, wlo); b <= std::min(L, whi); ++b) {
      const int64_t rem = (int64_t)r2 - (int64_t)a * a - (int64_t)b * b;
      if (rem < 0) continue;
      int w = (int)std::floor(std::sqrt((double)rem));
      while ((int64_t)w * w > rem) --w;
      while ((int64_t)(w + 1) * (w + 1) <= rem) ++w;
      cnt += std::min(w, whi) - std::max(-w, wlo) + 1;
    }
  return cnt;
}

#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      st = cuda_fail(e_, #x);                   \
      goto done;                                \
    }                                           \
  } while (0)

void free_sources(Grid& g) {
  Grid::Ingest& w = g.ing;
  dev_free(g.src); dev_free(g.ndot); dev_free(g.r2lim); dev_free(g.items);
  dev_free(g.src_of_input); dev_free(g.ndot_in);
  g.src = nullptr; g.ndot = nullptr; g.r2lim = nullptr; g.items = nullptr;
  g.src_of_input = nullptr; g.ndot_in = nullptr;
  g.src_cap = 0;
  dev_free(w.keys); dev_free(w.keys2); dev_free(w.idx); dev_free(w.idx2); dev_free(w.r2in);
  dev_free(w.head); dev_free(w.mid); dev_free(w.msrc); dev_free(w.mndot); dev_free(w.mr2);
  dev_free(w.lkey); dev_free(w.lkey2); dev_free(w.lval); dev_free(w.order); dev_free(w.lpt);
  dev_free(w.tmp); dev_free(w.dscal);
  cudaFreeHost(w.hscal); cudaFreeHost(w.r2pin); cudaFreeHost(w.srcpin);
  w = Grid::Ingest{};
}

// Grow the per-source arrays (ingest scratch and the ingested sources) to n sources.
static cudaError_t reserve_sources(Grid& g, size_t n) {
  Grid::Ingest& w = g.ing;
  if (n <= w.cap && n <= g.src_cap) return cudaSuccess;
  cudaStreamSynchronize(g.stream);  // earlier work may still read the old arrays
  free_sources(g);
  cudaError_t e = cudaSuccess;
  auto dm = [&](auto*& p, size_t bytes) {
    if (e == cudaSuccess) e = dev_malloc(reinterpret_cast<void**>(&p), bytes);
  };
  dm(w.keys, n * sizeof(uint64_t)); dm(w.keys2, n * sizeof(uint64_t));
  dm(w.idx, n * sizeof(int)); dm(w.idx2, n * sizeof(int)); dm(w.r2in, n * sizeof(int));
  dm(w.head, n * sizeof(int)); dm(w.mid, n * sizeof(int));
  dm(w.msrc, n * sizeof(SrcDev)); dm(w.mndot, n * sizeof(double)); dm(w.mr2, n * sizeof(int));
  dm(w.lkey, n * sizeof(uint32_t)); dm(w.lkey2, n * sizeof(uint32_t));
  dm(w.lval, n * sizeof(int)); dm(w.order, n * sizeof(int)); dm(w.lpt, n * sizeof(int));
  dm(w.dscal, 4 * sizeof(int));
  dm(g.src, n * sizeof(SrcDev)); dm(g.ndot, n * sizeof(double)); dm(g.r2lim, n * sizeof(int));
  dm(g.items, 24 * n * sizeof(int)); dm(g.src_of_input, n * sizeof(int));
  dm(g.ndot_in, n * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&w.hscal), 4 * sizeof(int));
  if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&w.r2pin), n * sizeof(int));
  if (e == cudaSuccess && g.nbox > 1)
    e = cudaMallocHost(reinterpret_cast<void**>(&w.srcpin), n * sizeof(SrcDev));
  // CUB scratch for the largest of its three uses at n items
  size_t need = 0, tb = 0;
  if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(nullptr, need, w.keys, w.keys2, w.idx,
                                                            w.idx2, (int)n, 0, 64, g.stream);
  tb = std::max(tb, need);
  if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(nullptr, need, w.head, w.mid, (int)n,
                                                          g.stream);
  tb = std::max(tb, need);
  if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(nullptr, need, w.lkey, w.lkey2, w.lval,
                                                            w.order, (int)n, 0, 32, g.stream);
  tb = std::max(tb, need);
  if (e == cudaSuccess) e = cub::DeviceReduce::Max(nullptr, need, w.r2in, w.dscal, (int)n,
                                                   g.stream);
  tb = std::max(tb, need);
  dm(w.tmp, tb);
  if (e != cudaSuccess) {
    free_sources(g);
    return e;
  }
  w.tmp_bytes = tb;
  w.cap = n;
  g.src_cap = n;
  return cudaSuccess;
}

rt_status ingest_sources(Grid& g, int nsrc, const int32_t* d_pos, const int32_t* d_box,
                         const double* d_ndot, const double* d_radius) {
  rt_status st = RT_OK;
  cudaStream_t s = g.stream;
  Grid::Ingest& w = g.ing;
  size_t need = 0;
  int nm = 0;
  const int T = 256;
  const int nb = (nsrc + T - 1) / T;

  g.nsrc = 0; g.nsrc_in = 0; g.max_r2 = 0; g.source_voxels = 0; g.r2_sorted_h.clear();
  if (nsrc == 0) return RT_OK;
  CK(reserve_sources(g, (size_t)nsrc));

  CK(cudaMemsetAsync(g.err + 1, 0, sizeof(int), s));  // the validation word, not the trace's
  k_src_keys<<<nb, T, 0, s>>>(g.boxes_d, g.nbox, nsrc, d_pos, d_box, d_ndot, d_radius, w.keys,
                              w.idx, w.r2in, g.err + 1);
  count_launch();
  CK(cudaGetLastError());
  // stable sort by (cell, r2): co-located sources with equal radius become adjacent
  // (keys of invalid sources are harmless: they are reported below before any use)
  need = w.tmp_bytes;
  CK(cub::DeviceRadixSort::SortPairs(w.tmp, need, w.keys, w.keys2, w.idx, w.idx2, nsrc, 0, 64, s));
  k_src_heads<<<nb, T, 0, s>>>(w.keys2, nsrc, w.head);
  count_launch();
  CK(cudaGetLastError());
  need = w.tmp_bytes;
  CK(cub::DeviceScan::ExclusiveSum(w.tmp, need, w.head, w.mid, nsrc, s));
  need = w.tmp_bytes;
  CK(cub::DeviceReduce::Max(w.tmp, need, w.r2in, w.dscal, nsrc, s));  // for the LPT key
  CK(cudaMemcpyAsync(w.hscal + 0, g.err + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(w.hscal + 1, w.head + nsrc - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(w.hscal + 2, w.mid + nsrc - 1, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(w.hscal + 3, w.dscal, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (w.hscal[0]) {
    st = fail(RT_ERR_INVALID, "rt_set_sources: source outside its box, bad box id, radius <= 0 "
                              "or non-finite/negative photon rate");
    goto done;
  }
  nm = w.hscal[2] + w.hscal[1];
  g.max_r2 = w.hscal[3];
  CK(cudaMemcpyAsync(g.ndot_in, d_ndot, nsrc * sizeof(double), cudaMemcpyDeviceToDevice, s));
  k_src_merge<<<nb, T, 0, s>>>(w.keys2, w.idx2, w.head, w.mid, nsrc, d_pos, d_box, d_ndot, w.r2in,
                               w.msrc, w.mndot, w.mr2, w.lkey, w.lval, g.src_of_input, g.max_r2);
  count_launch();
  CK(cudaGetLastError());
  need = w.tmp_bytes;
  CK(cub::DeviceRadixSort::SortPairs(w.tmp, need, w.lkey, w.lkey2, w.lval, w.order, nm, 0, 32, s));
  k_src_order<<<(nm + T - 1) / T, T, 0, s>>>(w.order, nm, w.msrc, w.mndot, w.mr2, g.src, g.ndot,
                                             g.r2lim, g.items, w.lpt);
  count_launch();
  CK(cudaGetLastError());
  k_remap<<<nb, T, 0, s>>>(g.src_of_input, w.lpt, nsrc);
  count_launch();
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(w.r2pin, g.r2lim, nm * sizeof(int), cudaMemcpyDeviceToHost, s));
  if (g.nbox > 1)
    CK(cudaMemcpyAsync(w.srcpin, g.src, nm * sizeof(SrcDev), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  {
    g.r2_sorted_h.assign(w.r2pin, w.r2pin + nm);
    std::map<std::pair<int, int>, int64_t>& memo = g.ball_memo;  // kept between calls
    int64_t sv = 0, last_cnt = 0;
    std::pair<int, int> last_key(-1, -1);
    for (int p = 0; p < nm; ++p) {  // sources come sorted by r2: runs of equal keys
      const int box = g.nbox > 1 ? w.srcpin[p].box : 0;
      const auto key = std::make_pair(g.r2_sorted_h[p], g.boxes_h[box].n);
      if (key != last_key) {
        auto it = memo.find(key);
        if (it == memo.end()) it = memo.emplace(key, ball_count(key.first, key.second)).first;
        last_key = key;
        last_cnt = it->second;
      }
      sv += last_cnt;
    }
    g.source_voxels = sv;
  }
  g.nsrc = nm;
  g.nsrc_in = nsrc;
done:
  return st;
}

// ------------------------------------------------------------ row tables
// Row tables of the unclipped quadrant layers of every distinct R^2 limit: the
// batched trace stages them into shared memory instead of building them per
// item (all 24 items of a source, and all sources with the same limit, share
// them).  Blob of (r2, m): rowpre[0..H+1] (ints: first flat index of row a1,
// then the layer size) and rowof[0..total) (bytes: row of every flat index),
// with H = min(m, isqrt(r2 - m^2)) and row a1 holding a2 = 0..min(H,
// isqrt(r2 - m^2 - a1^2)).
static int isqrt_host(int64_t x) {
  if (x < 0) return -1;
  int r = (int)std::sqrt((double)x);
  while ((int64_t)r * r > x) --r;
  while ((int64_t)(r + 1) * (r + 1) <= x) ++r;
  return r;
}

__global__ void k_row_tables(const int* __restrict__ ent_r2, const int* __restrict__ ent_m,
                             const int* __restrict__ off, unsigned char* __restrict__ rtab,
                             int nent) {
  const int e = blockIdx.x;
  if (e >= nent) return;
  const int m = ent_m[e];
  const int rem = ent_r2[e] - m * m;
  int H = (int)sqrtf((float)rem);
  while (H * H > rem) --H;
  while ((H + 1) * (H + 1) <= rem) ++H;
  H = min(H, m);
  const int nrows = H + 1;
  int* rowpre = reinterpret_cast<int*>(rtab + off[e]);
  unsigned char* rowof = reinterpret_cast<unsigned char*>(rowpre + nrows + 1);
  __shared__ int pre[256 + 1];
  if (threadIdx.x == 0) {
    int run = 0;
    for (int r = 0; r < nrows; ++r) {
      pre[r] = run;
      const int x = rem - r * r;
      int w = (int)sqrtf((float)x);
      while (w * w > x) --w;
      while ((w + 1) * (w + 1) <= x) ++w;
      run += min(H, w) + 1;
    }
    pre[nrows] = run;
  }
  __syncthreads();
  for (int r = threadIdx.x; r <= nrows; r += blockDim.x) rowpre[r] = pre[r];
  for (int r = 0; r < nrows; ++r)
    for (int c = pre[r] + threadIdx.x; c < pre[r + 1]; c += blockDim.x) rowof[c] = (unsigned char)r;
  // zero the padding up to the next 16-byte boundary
  const int used = 4 * (nrows + 1) + pre[nrows];
  for (int b = used + threadIdx.x; b < off[e + 1] - off[e]; b += blockDim.x)
    rtab[off[e] + b] = 0;
}

// Interior row tables of the same layers, for faces traced whole by one warp:
// layer m of a face holds the transverse offsets |t1|, |t2| <= H with
// t1^2 + t2^2 <= r2 - m^2; its interior positions (1 <= a1, a2 <= m-1) form rows
// a1 = 1..LA, LA = min(H, m-1), row a1 holding a2 = 1..min(H, isqrt(r2 - m^2 -
// a1^2), m-1).  Blob: rowpre[0..LA] (ints: first flat index of row r = a1-1,
// then the number of positions) and rowof[0..total) (bytes: row of every flat
// index).  The axes and the rim of the layer are enumerated arithmetically.
__device__ __forceinline__ int isqrt_dev(int x) {
  int w = (int)sqrtf((float)x);
  while (w * w > x) --w;
  while ((w + 1) * (w + 1) <= x) ++w;
  return w;
}

__global__ void k_interior_tables(const int* __restrict__ ent_r2, const int* __restrict__ ent_m,
                                  const int* __restrict__ off, unsigned char* __restrict__ itab,
                                  int nent) {
  const int e = blockIdx.x;
  if (e >= nent) return;
  const int m = ent_m[e];
  const int rem = ent_r2[e] - m * m;
  const int H = min(isqrt_dev(rem), m);
  const int LA = min(H, m - 1);
  int* rowpre = reinterpret_cast<int*>(itab + off[e]);
  unsigned char* rowof = reinterpret_cast<unsigned char*>(rowpre + LA + 1);
  __shared__ int pre[256 + 1];
  if (threadIdx.x == 0) {
    int run = 0;
    for (int r = 0; r < LA; ++r) {
      pre[r] = run;
      const int a1 = r + 1;
      run += max(0, min(min(H, isqrt_dev(rem - a1 * a1)), m - 1));
    }
    pre[LA] = run;
  }
  __syncthreads();
  for (int r = threadIdx.x; r <= LA; r += blockDim.x) rowpre[r] = pre[r];
  for (int r = 0; r < LA; ++r)
    for (int c = pre[r] + threadIdx.x; c < pre[r + 1]; c += blockDim.x) rowof[c] = (unsigned char)r;
  const int used = 4 * (LA + 1) + pre[LA];
  for (int b = used + threadIdx.x; b < off[e + 1] - off[e]; b += blockDim.x)
    itab[off[e] + b] = 0;
}

void free_row_tables(Grid& g) {
  dev_free(g.rtab); dev_free(g.rtab_off); dev_free(g.rtab_first); dev_free(g.rtab_hcap);
  dev_free(g.rtab_slot); dev_free(g.itab); dev_free(g.itab_off);
  g.rtab = nullptr; g.rtab_off = g.rtab_first = g.rtab_hcap = g.rtab_slot = nullptr;
  g.itab = nullptr; g.itab_off = nullptr;
  g.itab_bytes = 0;
  g.rtab_max_r2 = -1;
  g.rtab_bytes = 0;
  g.rtab_r2s.clear();
  g.rtab_mcap = 0;
}

rt_status ensure_row_tables(Grid& g) {
  rt_status st = RT_OK;
  // distinct limits, descending (r2_sorted_h is in LPT order: descending)
  std::vector<int> r2s;
  for (int v : g.r2_sorted_h)
    if (r2s.empty() || v != r2s.back()) r2s.push_back(v);
  std::sort(r2s.begin(), r2s.end(), std::greater<int>());
  r2s.erase(std::unique(r2s.begin(), r2s.end()), r2s.end());
  const int mcap = g.nmax / 2 + 1;  // no window has more layers
  if (r2s == g.rtab_r2s && mcap == g.rtab_mcap && (g.rtab || r2s.empty())) return RT_OK;
  free_row_tables(g);
  if (r2s.empty()) {
    g.rtab_mcap = mcap;
    return RT_OK;
  }
  std::vector<int> ent_r2, ent_m, off, ioff, first(r2s.size()), hcap(r2s.size());
  int64_t cur = 0, icur = 0;
  for (size_t i = 0; i < r2s.size(); ++i) {
    const int v = r2s[i];
    const int L = std::min(isqrt_host(v), mcap);
    first[i] = (int)ent_m.size();
    int hc = 0;
    for (int m = 1; m <= L; ++m) {
      const int64_t rem = (int64_t)v - (int64_t)m * m;
      const int H = std::min(m, isqrt_host(rem));
      int64_t total = 0;
      for (int r = 0; r <= H; ++r) total += std::min(H, isqrt_host(rem - (int64_t)r * r)) + 1;
      const int LA = std::min(H, m - 1);
      int64_t itotal = 0;
      for (int a1 = 1; a1 <= LA; ++a1)
        itotal += std::max(0, std::min(std::min(H, isqrt_host(rem - (int64_t)a1 * a1)), m - 1));
      hc = std::max(hc, H);
      ent_r2.push_back(v);
      ent_m.push_back(m);
      off.push_back((int)cur);
      ioff.push_back((int)icur);
      cur += (4 * (int64_t)(H + 2) + total + 15) & ~(int64_t)15;
      icur += (4 * (int64_t)(LA + 1) + itotal + 15) & ~(int64_t)15;
      if (cur > (int64_t)1 << 30 || H > 254) {  // keep offsets in int, rows in bytes
        g.rtab_r2s = r2s;
        g.rtab_mcap = mcap;
        return RT_OK;  // no tables: the trace builds its own
      }
    }
    hcap[i] = hc;
  }
  off.push_back((int)cur);
  ioff.push_back((int)icur);
  const int nent = (int)ent_m.size();
  const int maxv = r2s.front();
  std::vector<int> slot(maxv + 1, -1);
  for (size_t i = 0; i < r2s.size(); ++i) slot[r2s[i]] = (int)i;
  int *d_r2 = nullptr, *d_m = nullptr;
  cudaStream_t s = g.stream;
#undef CK
#define CK(x)                                   \
  do {                                          \
    cudaError_t e_ = (x);                       \
    if (e_ != cudaSuccess) {                    \
      st = cuda_fail(e_, #x);                   \
      goto fail;                                \
    }                                           \
  } while (0)
  CK(dev_malloc(&g.rtab, std::max<int64_t>(cur, 16)));
  CK(dev_malloc(&g.rtab_off, off.size() * sizeof(int)));
  CK(dev_malloc(&g.rtab_first, first.size() * sizeof(int)));
  CK(dev_malloc(&g.rtab_hcap, hcap.size() * sizeof(int)));
  CK(dev_malloc(&g.rtab_slot, slot.size() * sizeof(int)));
  CK(dev_malloc(&g.itab, std::max<int64_t>(icur, 16)));
  CK(dev_malloc(&g.itab_off, ioff.size() * sizeof(int)));
  CK(cudaMemcpyAsync(g.itab_off, ioff.data(), ioff.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(dev_malloc(&d_r2, std::max(nent, 1) * sizeof(int)));
  CK(dev_malloc(&d_m, std::max(nent, 1) * sizeof(int)));
  CK(cudaMemcpyAsync(g.rtab_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.rtab_first, first.data(), first.size() * sizeof(int),
                     cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.rtab_hcap, hcap.data(), hcap.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(g.rtab_slot, slot.data(), slot.size() * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_r2, ent_r2.data(), nent * sizeof(int), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(d_m, ent_m.data(), nent * sizeof(int), cudaMemcpyHostToDevice, s));
  if (nent > 0) {
    k_row_tables<<<nent, 64, 0, s>>>(d_r2, d_m, g.rtab_off, g.rtab, nent);
    count_launch();
    CK(cudaGetLastError());
    k_interior_tables<<<nent, 64, 0, s>>>(d_r2, d_m, g.itab_off, g.itab, nent);
    count_launch();
    CK(cudaGetLastError());
  }
  CK(cudaStreamSynchronize(s));  // host vectors go out of scope
  dev_free(d_r2);
  dev_free(d_m);
  g.rtab_max_r2 = maxv;
  g.rtab_bytes = cur;
  g.itab_bytes = icur;
  g.rtab_r2s = r2s;
  g.rtab_mcap = mcap;
  return RT_OK;
fail:
  cudaStreamSynchronize(s);
  dev_free(d_r2);
  dev_free(d_m);
  free_row_tables(g);
  return st;
#undef CK
}

}  // namespace asora
