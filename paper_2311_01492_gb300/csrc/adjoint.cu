// Adjoint of the ray trace: gradients of L = sum_p w_p Gamma_p with respect to
// log n_HI of every cell and log Ndot of every source.
//
// The forward recurrence of one (source, face) item (trace.cu) is
//   tau_in(p)  = sum_n w_n(p) tau_out(e_n(p))      (m >= 2; m = 1: dtau(s)/2 ds(p))
//   tau_out(p) = tau_in(p) + dtau(p) ds(p)
//   Gamma_sp   = Ndot [g(tau_in) - g(tau_out)] / (n_HI V)  or  Ndot sigma0 h(tau_in)/(4 pi r^2)
// so with lambda(p) = dL/dtau_out(p) and mu(p) = dL/dtau_in(p):
//   lambda(p) = w_p dGamma_sp/dtau_out + sum_{q uses p} w_n(q) mu(q)
//   mu(p)     = lambda(p) + w_p dGamma_sp/dtau_in
//   dL/dlog n_HI(p) += dtau(p) ds(p) lambda(p) - w_p Gamma_sp   (the last term: thick, 1/n_HI)
//   dL/ddtau(s)     += sum_{m=1 cells} mu(p) ds(p)/2 + lambda(s)/2
//   dL/dlog Ndot_s   = sum_p w_p Gamma_sp                         (Gamma is linear in Ndot)
// The users q of p lie in the next layer of the same face.  Each face seeds
// the adjoint with the direct terms of the cells it owns and propagates it
// through its whole closed pyramid, which contains the complete upstream cone
// of every cell in it; summing the faces' partial adjoints gives the total.
//
// Items are (source, face, quadrant) as in the batched trace.  Per item: a
// forward pass stores (tau_in, tau_out) of every layer in a per-CTA stack in
// global memory (the per-source column densities are never
// kept beyond the item), then a reverse pass walks the layers from the outside
// in with mu of the next layer in shared memory.  Built with --fmad=false.
#include <algorithm>
#include <cmath>

#include "asora_internal.cuh"
#include "device_util.cuh"

namespace asora {

// Stack capacity (double2) of one quadrant item for radius limit r2, box size n.
size_t face_stack_cap(int r2, int nmax) {
  size_t tot = 0;
  int L = (int)std::floor(std::sqrt((double)r2));
  while ((int64_t)L * L > r2) --L;
  L = std::min(L, nmax / 2 + 1);
  for (int m = 1; m <= L; ++m) {
    int h = (int)std::floor(std::sqrt((double)(r2 - m * m)));
    while (h > 0 && (int64_t)h * h > r2 - (int64_t)m * m) --h;
    h = std::min(h, m);
    tot += (size_t)(h + 1) * (h + 1);
  }
  return tot;
}

__host__ __device__ inline size_t r16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared memory of one adjoint group: two layers of (h+1)^2 doubles, one row
// table (h+2 ints, (h+1)^2 bytes), per-layer metadata (half-width, stack
// offset, "has rate cells" flag) for lcap layers, reduction scratch.
__host__ __device__ inline size_t bwd_group_bytes(int h, int lcap) {
  const size_t cap = (size_t)(h + 1) * (h + 1);
  return r16(2 * cap * sizeof(double)) + r16((size_t)(h + 2) * sizeof(int)) + r16(cap) +
         r16(2 * (size_t)(lcap + 2) * sizeof(int)) + r16((size_t)(lcap + 2)) + 64;
}

size_t bwd_smem_bytes(int hcap, int lcap) { return bwd_group_bytes(hcap, lcap); }

struct BwdArgs {
  TraceArgs t;
  const double* w;       // dL/dGamma per cell
  double* dlogn;         // dL/dlog n_HI per cell (accumulated)
  double* dndot;         // dL/dlog Ndot per merged source (accumulated)
  double2* stack;        // per-group (tau_in, tau_out) stacks
  size_t stack_cap;      // double2 per group
  int lcap;              // layer capacity of the metadata arrays
  int exit;              // stop the recompute at the first opaque layer (exact)
};

template <int GS>
__device__ __forceinline__ bool group_any(bool v) {
  if (GS == 32) {
    __syncwarp();
    return __any_sync(0xffffffffu, v);
  }
  return __syncthreads_or(v) != 0;
}

template <int GS>
__device__ __forceinline__ bool group_all(bool v) {
  if (GS == 32) {
    __syncwarp();
    return __all_sync(0xffffffffu, v);
  }
  return __syncthreads_and(v) != 0;
}

// Sum over the group; the result is valid in thread 0 of the group.
template <int GS>
__device__ __forceinline__ double group_sum(double v, double* red, int gt) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (GS == 32) return v;
  group_sync<GS>();
  if ((gt & 31) == 0) red[gt >> 5] = v;
  group_sync<GS>();
  double s = 0.0;
  if (gt == 0)
    for (int i = 0; i < GS / 32; ++i) s += red[i];
  return s;
}

// One (source, face, quadrant) item of the adjoint with a group of GS threads.
template <int GS>
__device__ __forceinline__ void bwd_item(const BwdArgs& A, const int item, const int gt,
                                         unsigned char* __restrict__ sm, double2* __restrict__ stk) {
  const TraceArgs& a = A.t;
  const int h = a.hcap;
  const int cap = (h + 1) * (h + 1);
  double* bufA = reinterpret_cast<double*>(sm);
  double* bufB = bufA + cap;
  unsigned char* p = sm + r16(2 * (size_t)cap * sizeof(double));
  int* rowpre = reinterpret_cast<int*>(p);
  p += r16((size_t)(h + 2) * sizeof(int));
  unsigned char* rowof = p;
  p += r16((size_t)cap);
  int* lH = reinterpret_cast<int*>(p);
  int* lO = lH + A.lcap + 2;
  p += r16(2 * (size_t)(A.lcap + 2) * sizeof(int));
  unsigned char* lnear = p;
  p += r16((size_t)(A.lcap + 2));
  double* red = reinterpret_cast<double*>(p);
  const int wid = gt >> 5, lane = gt & 31;

  const int s = item >> 5, f = (item >> 2) & 7, quad = item & 3;
  const SrcDev S = a.src[s];
  const BoxDev B = a.boxes[S.box];
  const int N = B.n;
  const int R2 = a.r2lim[s];
  const double nd = a.ndot[s];
  const int d = f >> 1;
  const int sg = (f & 1) ? -1 : 1;
  const int q1 = (quad & 1) ? -1 : 1, q2 = (quad & 2) ? -1 : 1;
  const int lim1 = q1 > 0 ? B.whi : -B.wlo, lim2 = q2 > 0 ? B.whi : -B.wlo;
  int Lmax = sg > 0 ? B.whi : -B.wlo;
  Lmax = min(Lmax, isqrt_i(R2));
  if (Lmax > A.lcap) {
    if (gt == 0) atomicOr(a.err, ERR_LAYER_CAP);
    return;
  }
  const int64_t scell = B.off + ((int64_t)S.i * N + S.j) * N + S.k;
  const double dts = a.dtau[scell];
  const int64_t NN = (int64_t)N * N;
  const int c1 = d == 0 ? S.j : S.i;
  const int c2 = d == 2 ? S.j : S.k;
  const int cd = d == 0 ? S.i : (d == 1 ? S.j : S.k);
  const int64_t m1 = d == 0 ? (int64_t)N : (d == 1 ? NN : (int64_t)N);
  const int64_t md = d == 0 ? NN : (d == 1 ? (int64_t)N : NN);
  const double* __restrict__ fld = (d == 2 ? a.dtauT : a.dtau) + B.off;
  double qacc = 0.0;    // sum_p w_p Gamma_sp over owned cells of this item
  double srcacc = 0.0;  // dL/ddtau(s) from this item

  // source cell (owned by face 4, quadrant 0): rate, its Ndot and tau_out adjoints
  double lam_s = 0.0, ndir_s = 0.0;
  if (f == 4 && quad == 0 && gt == 0) {
    const double tout = 0.5 * dts;
    const double ws = A.w[scell];
    if (bits_of(tout) <= bits_of(a.tau_lim)) {
      qacc += ws * (nd * (tab_eval(a.tab.h, a.tab, 0.0) * (0.5 * B.thin_fac)));
    } else {
      const double fct = nd * B.inv_cell3 * a.invn[scell];
      const double G = fct * (tab_eval(a.tab.g, a.tab, 0.0) - tab_eval(a.tab.g, a.tab, tout));
      qacc += ws * G;
      lam_s = -ws * fct * tab_slope(a.tab.g, a.tab, tout);
      ndir_s = -ws * G;
    }
  }

  // ------------------------------------------------ forward (recompute)
  double* prev = bufA;
  double* cur = bufB;
  int Hp = 0, Llast = 0;
  size_t off = 0;
  if (gt == 0) prev[0] = 0.5 * dts;  // the interpolant of every layer-1 cell
  for (int m = 1; m <= Lmax; ++m) {
    const int rem = R2 - m * m;
    const int H = min(m, isqrt_i(rem));
    const size_t W2 = (size_t)(H + 1) * (H + 1);
    if (H > h || m > a.geo_mmax || off + W2 > A.stack_cap) {
      if (gt == 0) atomicOr(a.err, ERR_LAYER_CAP);
      return;
    }
    if (gt == 0) {
      lH[m] = H;
      lO[m] = (int)off;
    }
    const int nrows = min(H, lim1) + 1;
    if (wid == 0) quad_rows_warp(rem, H, nrows, lim2, rowpre, rowof, lane);
    group_sync<GS>();
    const int total = rowpre[nrows];
    const int W = H + 1, Wp = Hp + 1;
    const int lc = wrapc(cd + sg * m, N);
    const int64_t lay = (int64_t)lc * md;
    const int gbase = (int)geo_index(m, 0, 0);
    bool near = false, opaque = true;
    for (int t = gt; t < total; t += GS) {
      const int a1 = rowof[t];
      const int a2 = t - rowpre[a1];
      const int x1 = wrapc(c1 + q1 * a1, N), x2 = wrapc(c2 + q2 * a2, N);
      const int64_t gidx = lay + x1 * m1 + x2;
      const double dtp = __ldg(&fld[gidx]);
      const GeoEntry* ge = &a.geo[gbase + ((max(a1, a2) * (max(a1, a2) + 1)) >> 1) + min(a1, a2)];
      const double ds = __ldg(&ge->ds);
      // Layer 1 (tau_in = (dtau_s/2) ds) goes through the same chain, so that no
      // branch on m turns into an FP64 product issued with every lane predicated
      // off in the other layers' rounds: its interpolants all read slot 0 of the
      // previous buffer, which holds dtau_s/2, with weights (ds, 0, 0, 0); the
      // zero terms add exactly +0.
      const bool l1 = m == 1;
      const double wa = __ldg(&ge->wa), wb = __ldg(&ge->wb);
      const double w1 = l1 ? ds : __ldg(&ge->w1), w4 = l1 ? 0.0 : __ldg(&ge->w4);
      const double w2 = l1 ? 0.0 : (a1 <= a2 ? wa : wb);
      const double w3 = l1 ? 0.0 : (a1 <= a2 ? wb : wa);
      const int b1 = min(a1, Hp), b2 = min(a1 - (a1 > 0), Hp);
      const int e1 = min(a2, Hp), e2 = min(a2 - (a2 > 0), Hp);
      const double tin = fma(w4, prev[b2 * Wp + e2],
                             fma(w3, prev[b1 * Wp + e2], fma(w2, prev[b2 * Wp + e1],
                                                             w1 * prev[b1 * Wp + e1])));
      const double tout = fma(dtp, ds, tin);
      const int li = a1 * W + a2;
      cur[li] = tout;
      stk[off + li] = make_double2(tin, tout);
      opaque = opaque && bits_of(tout) >= a.exit_bits;
      const bool rate = bits_of(tin) < a.tab.tau_max_bits;
      near = near || rate;
      const bool own = ((d == 2) || (d == 1 ? a2 < m : (a1 < m && a2 < m))) &&
                       (a1 > 0 || q1 > 0) && (a2 > 0 || q2 > 0);
      if (own && rate) {
        const int64_t cell = B.off + (d == 2 ? ((int64_t)x1 * N + x2) * N + lc : gidx);
        const double wp = __ldg(&A.w[cell]);
        if (wp != 0.0) {
          const double dcell = dtp * ds;
          double G;
          if (bits_of(dcell) <= bits_of(a.tau_lim))
            G = nd * (tab_eval(a.tab.h, a.tab, tin) * (__ldg(&ge->thin) * B.thin_fac));
          else
            G = nd * ((tab_eval(a.tab.g, a.tab, tin) - tab_eval(a.tab.g, a.tab, tout)) *
                      (__ldg(&ge->invv) * B.inv_cell3) * __ldg(&a.invn[cell]));
          qacc += wp * G;
        }
      }
    }
    const bool near_any = group_any<GS>(near);
    const bool all_opaque = group_all<GS>(opaque);
    if (gt == 0) lnear[m] = near_any ? 1 : 0;
    double* tmp = prev;
    prev = cur;
    cur = tmp;
    Hp = H;
    off += W2;
    Llast = m;
    // No rate beyond a fully opaque layer (every later tau_in >= 2^E1): the
    // adjoint gets nothing from the rest of the pyramid.
    if (A.exit && all_opaque) break;
  }
  group_sync<GS>();

  // ------------------------------------------------ reverse
  double* next = bufA;  // mu of layer m+1
  double* mu = bufB;    // mu of layer m
  int Hn = -1;
  bool nz_next = false;  // whether layer m+1 has any non-zero mu
  for (int m = Llast; m >= 1; --m) {
    const int H = lH[m];
    if (!nz_next && !lnear[m]) {
      // no adjoint arrives and no rate cell: mu = 0 and nothing to deposit here
      Hn = H;
      continue;
    }
    const int rem = R2 - m * m;
    const int W = H + 1, Wn = Hn + 1;
    for (int t = gt; t < W * W; t += GS) mu[t] = 0.0;
    const int nrows = min(H, lim1) + 1;
    if (wid == 0) quad_rows_warp(rem, H, nrows, lim2, rowpre, rowof, lane);
    group_sync<GS>();
    const int total = rowpre[nrows];
    const int lc = wrapc(cd + sg * m, N);
    const int64_t lay = (int64_t)lc * md;
    const int gbase = (int)geo_index(m, 0, 0);
    const int gnext = nz_next ? (int)geo_index(m + 1, 0, 0) : 0;
    const size_t o = (size_t)lO[m];
    bool nz = false;
    for (int t = gt; t < total; t += GS) {
      const int a1 = rowof[t];
      const int a2 = t - rowpre[a1];
      const int li = a1 * W + a2;
      // users of p in layer m+1 of this quadrant: (a1 | a1+1, a2 | a2+1); the
      // +1 ones step back onto p along that axis
      double lam = 0.0;
      if (nz_next) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const int u = a1 + i;
          if (u > Hn) continue;
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const int v = a2 + j;
            if (v > Hn) continue;
            const double muq = next[u * Wn + v];
            if (muq == 0.0) continue;
            const GeoEntry* gq = &a.geo[gnext + ((max(u, v) * (max(u, v) + 1)) >> 1) + min(u, v)];
            double wq;
            if (i == 0 && j == 0) wq = __ldg(&gq->w1);
            else if (i == 1 && j == 1) wq = __ldg(&gq->w4);
            else if (i == 1) wq = u <= v ? __ldg(&gq->wa) : __ldg(&gq->wb);  // w2(q)
            else wq = u <= v ? __ldg(&gq->wb) : __ldg(&gq->wa);              // w3(q)
            lam = fma(wq, muq, lam);
          }
        }
      }
      double2 tt = make_double2(0.0, 0.0);
      bool rate = false;
      if (lnear[m]) {
        tt = stk[o + li];
        rate = bits_of(tt.x) < a.tab.tau_max_bits;
      }
      if (lam == 0.0 && !rate) continue;  // mu = 0 (zeroed) and nothing to deposit
      const double tin = tt.x, tout = tt.y;
      const bool own = ((d == 2) || (d == 1 ? a2 < m : (a1 < m && a2 < m))) &&
                       (a1 > 0 || q1 > 0) && (a2 > 0 || q2 > 0);
      const int x1 = wrapc(c1 + q1 * a1, N), x2 = wrapc(c2 + q2 * a2, N);
      const int64_t gidx = lay + x1 * m1 + x2;
      const int64_t cell = B.off + (d == 2 ? ((int64_t)x1 * N + x2) * N + lc : gidx);
      const GeoEntry* ge = &a.geo[gbase + ((max(a1, a2) * (max(a1, a2) + 1)) >> 1) + min(a1, a2)];
      const double ds = __ldg(&ge->ds);
      const double dtp = __ldg(&fld[gidx]);
      // lam: dL/dtau_out(p); mup: dL/dtau_in(p) = lam + w dGamma/dtau_in.  In the
      // thick form the two direct terms are combined as the slope difference
      // g'(tau_in) - g'(tau_out) (0 within one chord segment) before adding.
      double mup = lam, ndir = 0.0;
      if (own && rate) {
        const double wp = __ldg(&A.w[cell]);
        if (wp != 0.0) {
          const double dcell = dtp * ds;
          if (bits_of(dcell) <= bits_of(a.tau_lim)) {
            mup = lam + wp * (nd * (tab_slope(a.tab.h, a.tab, tin) * (__ldg(&ge->thin) * B.thin_fac)));
          } else {
            const double fct = nd * (__ldg(&ge->invv) * B.inv_cell3) * __ldg(&a.invn[cell]);
            const double G = fct * (tab_eval(a.tab.g, a.tab, tin) - tab_eval(a.tab.g, a.tab, tout));
            const double si = tab_slope(a.tab.g, a.tab, tin), so = tab_slope(a.tab.g, a.tab, tout);
            mup = lam + (wp * fct) * (si - so);
            lam = lam - (wp * fct) * so;
            ndir = -wp * G;
          }
        }
      }
      mu[li] = mup;
      nz = nz || mup != 0.0;
      const double contrib = dtp * (lam * ds) + ndir;
      if (contrib != 0.0) atomicAdd(&A.dlogn[cell], contrib);
    }
    if (m == 1) {
      // dL/ddtau(s) from layer 1, after its rounds (kept out of the cell loop so that
      // no FP64 product runs with every lane off in the other layers): the same
      // thread takes the same cells as in the loop, so each partial sum is unchanged
      for (int t = gt; t < total; t += GS) {
        const int a1 = rowof[t];
        const int a2 = t - rowpre[a1];
        const GeoEntry* ge = &a.geo[gbase + ((max(a1, a2) * (max(a1, a2) + 1)) >> 1) + min(a1, a2)];
        const double mup = mu[a1 * W + a2];
        if (!(bits_of(mup) << 1)) continue;  // mu = 0: no term (as in the loop)
        srcacc += mup * (0.5 * __ldg(&ge->ds));
      }
    }
    nz_next = group_any<GS>(nz);
    double* tmp = next;
    next = mu;
    mu = tmp;
    Hn = H;
  }
  // per-item reductions: dL/dlog Ndot and the source cell's dtau adjoint
  const double qsum = group_sum<GS>(qacc, red, gt);
  const double ssum = group_sum<GS>(srcacc, red, gt);
  if (gt == 0) {
    if (qsum != 0.0) atomicAdd(&A.dndot[s], qsum);
    const double cs = dts * (ssum + 0.5 * lam_s) + ndir_s;
    if (cs != 0.0) atomicAdd(&A.dlogn[scell], cs);
  }
  group_sync<GS>();
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK, 6) k_trace_faces_bwd(BwdArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  const TraceArgs& a = A.t;
  if (a.skip && *a.skip) return;
  double2* stk = A.stack + (size_t)blockIdx.x * A.stack_cap;
  const int cap = (a.hcap + 1) * (a.hcap + 1);
  double* buf = reinterpret_cast<double*>(smem_raw);
  for (int t = threadIdx.x; t < 2 * cap; t += BLOCK) buf[t] = 0.0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = a.item_begin + atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) break;
    bwd_item<BLOCK>(A, a.items[it], threadIdx.x, smem_raw, stk);
  }
}

template <int WPB>
__global__ void __launch_bounds__(WPB * 32, 2) k_trace_faces_bwd_warp(BwdArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TraceArgs& a = A.t;
  if (a.skip && *a.skip) return;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* my = smem_raw + (size_t)wid * bwd_group_bytes(a.hcap, A.lcap);
  double2* stk = A.stack + ((size_t)blockIdx.x * WPB + wid) * A.stack_cap;
  const int cap = (a.hcap + 1) * (a.hcap + 1);
  double* buf = reinterpret_cast<double*>(my);
  for (int t = lane; t < 2 * cap; t += 32) buf[t] = 0.0;
  __syncwarp();
  for (;;) {
    int it = 0;
    if (lane == 0) it = a.item_begin + atomicAdd(a.queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= a.n_items) break;
    bwd_item<32>(A, a.items[it], lane, my, stk);
  }
}

constexpr int kBwdBlock = 128;
constexpr int kBwdWarps = 8;

// block 32: warp mode (kBwdWarps warps per CTA, one stack per warp).
cudaError_t launch_trace_bwd(Grid& g, const TraceArgs& t, const double* w, double* dlogn,
                             double* dndot_merged, double2* stack, size_t stack_cap, int lcap,
                             int grid, size_t smem, int block, bool exit) {
  BwdArgs A;
  A.t = t;
  A.w = w;
  A.dlogn = dlogn;
  A.dndot = dndot_merged;
  A.stack = stack;
  A.stack_cap = stack_cap;
  A.lcap = lcap;
  A.exit = exit ? 1 : 0;
  const void* fn = block == 32 ? (const void*)k_trace_faces_bwd_warp<kBwdWarps>
                               : (const void*)k_trace_faces_bwd<kBwdBlock>;
  const int threads = block == 32 ? kBwdWarps * 32 : kBwdBlock;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* params[] = {&A};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), params, smem, g.stream);
  count_launch();
  return e;
}

int bwd_max_grid(size_t smem, int block) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = block == 32 ? (const void*)k_trace_faces_bwd_warp<kBwdWarps>
                               : (const void*)k_trace_faces_bwd<kBwdBlock>;
  const int threads = block == 32 ? kBwdWarps * 32 : kBwdBlock;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
  if (e != cudaSuccess) return 0;
  return per * sms;
}

// dL/dlog Ndot of each input source from its merged source: Gamma is linear in
// the merged rate, so each member gets its share.
__global__ void k_dndot_inputs(int nsrc, const int* __restrict__ src_of_input,
                               const double* __restrict__ ndot_in,
                               const double* __restrict__ ndot_merged,
                               const double* __restrict__ dmerged, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsrc) return;
  const int m = src_of_input[i];
  const double nm = ndot_merged[m];
  out[i] = nm > 0.0 ? (ndot_in[i] / nm) * dmerged[m] : 0.0;
}

cudaError_t launch_dndot_inputs(Grid& g, const double* dmerged, double* out) {
  const int T = 256;
  k_dndot_inputs<<<(g.nsrc_in + T - 1) / T, T, 0, g.stream>>>(g.nsrc_in, g.src_of_input,
                                                               g.ndot_in, g.ndot, dmerged, out);
  count_launch();
  return cudaGetLastError();
}

}  // namespace asora
