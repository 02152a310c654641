// Short-characteristics ray tracing kernels (arXiv 2311.01492, Sec. 3.1-3.3).
//
// Both kernels evaluate, for every traced cell p of a source s, the same FP64
// recurrence with the same roundings (no implicit contraction: this file is
// built with --fmad=false; every fused multiply-add is an explicit fma()):
//
//   m = max|Delta|, weights W (geometry table), ds (geometry table)
//   tau_in  = fma(w4,c4, fma(w3,c3, fma(w2,c2, w1*c1)))   (Eq. interp)
//           = (dtau(s)/2)*ds                              if m == 1
//   tau_out = fma(dtau(p), ds, tau_in)
//   Gamma(p) += Ndot [g(tau_in) - g(tau_out)] / (n_HI V)   (Eq. sugg), or the
//               thin limit Ndot sigma0 h(tau_in)/(4 pi r^2) if dtau*ds <= tau_lim.
//
// k_trace_shells (RT_SCHED_PLAIN) follows ASORA's own schedule (Sec. 3.3,
// App. A): one CTA per source walks the octahedral shells S_q, q = 0..Q, with
// a CTA-wide barrier between shells, keeping the column densities of its
// source in a private cube of global memory.
//
// k_trace_faces (RT_SCHED_BATCHED) is the GB300 schedule.  The interpolants of
// a cell whose dominant axis is d lie in the plane one step closer to the
// source along d (Eq. raga, entry plane), so the cells with dominant axis d
// and sign +-1 -- a square pyramid ("face") -- form layers m = 1, 2, ... that
// each depend only on the previous layer of the same face.  A tie cell
// (|Delta_d| equal to another |Delta|) gets the same value from every face
// that contains it, because the weights of its out-of-face interpolants are
// exactly zero; each face therefore traces its closed pyramid independently
// and only the owning face (k before j before i) deposits the rate.  The six
// faces of every source are independent work items taken longest-first from
// a device queue by persistent CTAs; each layer lives in shared memory (two
// buffers of (2H+1)^2 doubles), so a cell reads only the previous layer.
#include <algorithm>
#include <cmath>

#include "asora_internal.cuh"

namespace asora {

__device__ __forceinline__ int isqrt_i(int x) {
  int r = (int)sqrtf((float)x);
  while (r * r > x) --r;
  while ((r + 1) * (r + 1) <= x) ++r;
  return r;
}

__device__ __forceinline__ int wrapc(int x, int n) {
  x = x < 0 ? x + n : x;
  return x >= n ? x - n : x;
}

__device__ __forceinline__ int sgn_i(int x) { return (x > 0) - (x < 0); }

__device__ __forceinline__ uint64_t bits_of(double x) {
  return (uint64_t)__double_as_longlong(x);
}

// Chord table lookup: segment from the IEEE bits of tau (tau >= +0).
__device__ __forceinline__ double tab_eval(const double2* __restrict__ t, const TabDev& tb,
                                           double tau) {
  if (tb.kind == RT_TABLE_GREY_EXACT) return exp(-tau);
  const uint64_t b = bits_of(tau);
  if (b >= tb.tau_max_bits) return 0.0;
  int seg = 0;
  if (b >= tb.tau_min_bits) {
    const int e = (int)(b >> 52) - 1023;
    const int m = (int)((b >> (52 - tb.B)) & (uint64_t)((1 << tb.B) - 1));
    seg = 1 + ((e + tb.E0) << tb.B) + m;
  }
  const double2 c = __ldg(&t[seg]);
  return fma(c.y, tau, c.x);
}

// Rate of one cell (photon-conserving, Eq. sugg; thin limit Eq. gammalocal).
__device__ __forceinline__ double cell_rate(const TraceArgs& a, double nd, double tin, double tout,
                                            double dcell, double invv_cell, double thin_cell,
                                            double invn) {
  if (bits_of(dcell) <= bits_of(a.tau_lim)) {
    return nd * (tab_eval(a.tab.h, a.tab, tin) * thin_cell);
  }
  const double dg = tab_eval(a.tab.g, a.tab, tin) - tab_eval(a.tab.g, a.tab, tout);
  return nd * (dg * invv_cell * invn);
}

// ----------------------------------------------------------- face kernel
size_t faces_smem_bytes(int hcap, int /*block*/) {
  const size_t cap = (size_t)(2 * hcap + 1) * (2 * hcap + 1);
  return 2 * cap * sizeof(double) + (size_t)(2 * hcap + 4) * sizeof(int);
}

template <int BLOCK, bool COLDENS>
__global__ void __launch_bounds__(BLOCK) k_trace_faces(TraceArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  __shared__ int s_total;
  const int hcap = a.hcap;
  const int cap = (2 * hcap + 1) * (2 * hcap + 1);
  double* buf0 = reinterpret_cast<double*>(smem_raw);
  double* buf1 = buf0 + cap;
  int* rowpre = reinterpret_cast<int*>(buf1 + cap);
  const int tid = threadIdx.x;
  if (a.skip && *a.skip) return;
  for (int t = tid; t < 2 * cap; t += BLOCK) buf0[t] = 0.0;
  unsigned nrate = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) {
      if (a.rate_cells) {
        for (int o = 16; o > 0; o >>= 1) nrate += __shfl_down_sync(0xffffffffu, nrate, o);
        if ((tid & 31) == 0 && nrate) atomicAdd(a.rate_cells, (unsigned long long)nrate);
      }
      break;
    }
    const int item = a.items[it];
    const int s = item >> 3, f = item & 7;
    const SrcDev S = a.src[s];
    const BoxDev B = a.boxes[S.box];
    const int N = B.n;
    const int R2 = a.r2lim[s];
    const double nd = a.ndot[s];
    const int d = f >> 1;
    const int sg = (f & 1) ? -1 : 1;
    int Lmax = sg > 0 ? B.whi : -B.wlo;
    Lmax = min(Lmax, isqrt_i(R2));
    const int64_t scell = B.off + ((int64_t)S.i * N + S.j) * N + S.k;
    const double dts = a.dtau[scell];

    if (f == 4 && tid == 0) {  // the source cell (q = 0), once per source
      const double tout = 0.5 * dts;
      if (COLDENS) {
        a.coldens[scell] = tout / a.sigma0;
      } else {
        double dG;
        if (bits_of(tout) <= bits_of(a.tau_lim))
          dG = nd * (tab_eval(a.tab.h, a.tab, 0.0) * (0.5 * B.thin_fac));
        else
          dG = nd * ((tab_eval(a.tab.g, a.tab, 0.0) - tab_eval(a.tab.g, a.tab, tout)) *
                     B.inv_cell3 * a.invn[scell]);
        if (dG != 0.0) atomicAdd(&a.gamma[scell], dG);
      }
    }

    double* prev = buf0;
    double* cur = buf1;
    int Hp = 0;
    for (int m = 1; m <= Lmax; ++m) {
      const int rem = R2 - m * m;
      const int H = min(m, isqrt_i(rem));
      if (H > hcap) {
        if (tid == 0) atomicOr(a.err, ERR_LAYER_CAP);
        break;
      }
      if (m > a.geo_mmax) {
        if (tid == 0) atomicOr(a.err, ERR_GEO);
        break;
      }
      const int u0 = max(-H, B.wlo), u1 = min(H, B.whi);
      const int nrows = u1 - u0 + 1;
      if (tid < 32) {  // row lengths of the layer and their prefix sums
        const int per = (nrows + 31) >> 5;
        const int rb = tid * per, re = min(nrows, rb + per);
        int local = 0;
        for (int r = rb; r < re; ++r) {
          const int t1 = u0 + r;
          const int w = min(H, isqrt_i(rem - t1 * t1));
          local += min(w, B.whi) - max(-w, B.wlo) + 1;
        }
        int incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (tid >= o) incl += v;
        }
        int run = incl - local;
        for (int r = rb; r < re; ++r) {
          rowpre[r] = run;
          const int t1 = u0 + r;
          const int w = min(H, isqrt_i(rem - t1 * t1));
          run += min(w, B.whi) - max(-w, B.wlo) + 1;
        }
        if (tid == 31) s_total = incl;
      }
      __syncthreads();
      const int total = s_total;
      const int W = 2 * H + 1, Wp = 2 * Hp + 1;
      for (int t = tid; t < total; t += BLOCK) {
        int lo = 0, hi = nrows - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (rowpre[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const int t1 = u0 + lo;
        const int w = min(H, isqrt_i(rem - t1 * t1));
        const int t2 = max(-w, B.wlo) + (t - rowpre[lo]);
        int di, dj, dk;
        if (d == 2) { di = t1; dj = t2; dk = sg * m; }
        else if (d == 1) { di = t1; dj = sg * m; dk = t2; }
        else { di = sg * m; dj = t1; dk = t2; }
        const int ii = wrapc(S.i + di, N), jj = wrapc(S.j + dj, N), kk = wrapc(S.k + dk, N);
        const int64_t cell = B.off + ((int64_t)ii * N + jj) * N + kk;
        const double dtp = (d == 2) ? __ldg(&a.dtauT[B.off + ((int64_t)kk * N + ii) * N + jj])
                                    : __ldg(&a.dtau[cell]);
        const int at1 = abs(t1), at2 = abs(t2);
        const int glo = min(at1, at2), ghi = max(at1, at2);
        const GeoEntry* ge = &a.geo[geo_index(m, glo, ghi)];
        const double2 wv0 = __ldg(reinterpret_cast<const double2*>(ge));      // w1, wa
        const double2 wv1 = __ldg(reinterpret_cast<const double2*>(ge) + 1);  // wb, w4
        const double ds = __ldg(&ge->ds);
        const double w1 = wv0.x, w4 = wv1.y;
        const double w2 = at1 <= at2 ? wv0.y : wv1.x;
        const double w3 = at1 <= at2 ? wv1.x : wv0.y;
        double tin;
        if (m == 1) {
          tin = (0.5 * dts) * ds;
        } else {
          const int s1 = sgn_i(t1), s2 = sgn_i(t2);
          const int a1 = min(max(t1, -Hp), Hp) + Hp, a2 = min(max(t1 - s1, -Hp), Hp) + Hp;
          const int b1 = min(max(t2, -Hp), Hp) + Hp, b2 = min(max(t2 - s2, -Hp), Hp) + Hp;
          const double c1 = prev[a1 * Wp + b1];
          const double c2 = prev[a2 * Wp + b1];
          const double c3 = prev[a1 * Wp + b2];
          const double c4 = prev[a2 * Wp + b2];
          tin = fma(w4, c4, fma(w3, c3, fma(w2, c2, w1 * c1)));
        }
        const double tout = fma(dtp, ds, tin);
        cur[(t1 + H) * W + (t2 + H)] = tout;
        const bool own = (d == 2) || (d == 1 ? at2 < m : (at1 < m && at2 < m));
        if (COLDENS) {
          if (own) a.coldens[cell] = tout / a.sigma0;
        } else if (own && bits_of(tin) < a.tab.tau_max_bits) {
          const double dcell = dtp * ds;
          const double dG = cell_rate(a, nd, tin, tout, dcell, __ldg(&ge->invv) * B.inv_cell3,
                                      __ldg(&ge->thin) * B.thin_fac,
                                      bits_of(dcell) <= bits_of(a.tau_lim) ? 0.0 : __ldg(&a.invn[cell]));
          ++nrate;
          if (dG != 0.0) atomicAdd(&a.gamma[cell], dG);
        }
      }
      __syncthreads();
      double* tmp = prev;
      prev = cur;
      cur = tmp;
      Hp = H;
    }
  }
}

template <int BLOCK>
static cudaError_t launch_faces_t(const TraceArgs& a, int grid, size_t smem, cudaStream_t s,
                                  bool coldens) {
  cudaError_t e;
  if (coldens) {
    e = cudaFuncSetAttribute(k_trace_faces<BLOCK, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_trace_faces<BLOCK, true><<<grid, BLOCK, smem, s>>>(a);
    count_launch();
  } else {
    e = cudaFuncSetAttribute(k_trace_faces<BLOCK, false>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k_trace_faces<BLOCK, false><<<grid, BLOCK, smem, s>>>(a);
    count_launch();
  }
  return cudaGetLastError();
}

cudaError_t launch_trace_faces(Grid& g, const TraceArgs& a, int block, int grid, size_t smem) {
  const bool cd = a.coldens != nullptr;
  switch (block) {
    case 64: return launch_faces_t<64>(a, grid, smem, g.stream, cd);
    case 128: return launch_faces_t<128>(a, grid, smem, g.stream, cd);
    case 256: return launch_faces_t<256>(a, grid, smem, g.stream, cd);
    case 512: return launch_faces_t<512>(a, grid, smem, g.stream, cd);
    default: return cudaErrorInvalidValue;
  }
}

int faces_max_grid(int block, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
#define OCC(B)                                                                              \
  case B:                                                                                   \
    e = cudaFuncSetAttribute(k_trace_faces<B, false>,                                       \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
    if (e == cudaSuccess)                                                                   \
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_faces<B, false>, B, smem); \
    break;
  switch (block) {
    OCC(64)
    OCC(128)
    OCC(256)
    OCC(512)
    default: return 0;
  }
#undef OCC
  if (e != cudaSuccess) return 0;
  return per * sms;
}

// ---------------------------------------------------------- shell kernel
// Cell t of the octahedral shell S_q (|S_q| = 4q^2+2, Sec. 3.3): the top part
// (Dk >= 0) is the diamond |Di|+|Dj| <= q, the bottom part (Dk < 0) the
// diamond of radius q-1, with |Dk| = q - |Di| - |Dj|.  A diamond of radius r
// holds the points with a = Di+Dj, b = Di-Dj of equal parity and |a|,|b| <= r:
// (r+1)^2 points with a,b = r (mod 2) followed by r^2 with a,b = r+1 (mod 2).
__host__ __device__ inline void shell_cell(int q, int t, int& di, int& dj, int& dk) {
  const int top = 2 * q * q + 2 * q + 1;
  int r, u;
  bool up;
  if (t < top) { r = q; u = t; up = true; }
  else { r = q - 1; u = t - top; up = false; }
  int A, Bc, a, b;
  if (u < (r + 1) * (r + 1)) {
    A = u / (r + 1); Bc = u - A * (r + 1);
    a = -r + 2 * A; b = -r + 2 * Bc;
  } else {
    u -= (r + 1) * (r + 1);
    A = u / r; Bc = u - A * r;
    a = -r + 1 + 2 * A; b = -r + 1 + 2 * Bc;
  }
  di = (a + b) / 2;
  dj = (a - b) / 2;
  const int h = q - (di < 0 ? -di : di) - (dj < 0 ? -dj : dj);
  dk = up ? h : -h;
}

template <int BLOCK>
__global__ void __launch_bounds__(BLOCK) k_trace_shells(TraceArgs a) {
  __shared__ int s_item;
  const int E = a.hcap;
  const int side = 2 * E + 1;
  double* cube = a.scratch + (size_t)blockIdx.x * side * side * side;
  const int tid = threadIdx.x;
  if (a.skip && *a.skip) return;
  unsigned nrate = 0;
  auto cidx = [&](int x, int y, int z) {
    return ((size_t)(x + E) * side + (size_t)(y + E)) * side + (size_t)(z + E);
  };
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) {
      if (a.rate_cells) {
        for (int o = 16; o > 0; o >>= 1) nrate += __shfl_down_sync(0xffffffffu, nrate, o);
        if ((tid & 31) == 0 && nrate) atomicAdd(a.rate_cells, (unsigned long long)nrate);
      }
      break;
    }
    const int s = a.items ? a.items[it] : it;
    const SrcDev S = a.src[s];
    const BoxDev B = a.boxes[S.box];
    const int N = B.n;
    const int R2 = a.r2lim[s];
    const double nd = a.ndot[s];
    const int64_t scell = B.off + ((int64_t)S.i * N + S.j) * N + S.k;
    const double dts = a.dtau[scell];
    const int rmax = isqrt_i(R2);
    const int emax = min(rmax, max(-B.wlo, B.whi));
    if (emax > E) {
      if (tid == 0) atomicOr(a.err, ERR_CUBE);
      continue;
    }
    // |Delta|_1 <= sqrt(3) |Delta|_2: no traced cell lies beyond shell floor(sqrt(3 R2))
    const int Q = min(3 * emax, isqrt_i(3 * R2));
    for (int q = 0; q <= Q; ++q) {
      const int cnt = q == 0 ? 1 : 4 * q * q + 2;
      for (int t = tid; t < cnt; t += BLOCK) {
        int di, dj, dk;
        shell_cell(q, t, di, dj, dk);
        if (di < B.wlo || di > B.whi || dj < B.wlo || dj > B.whi || dk < B.wlo || dk > B.whi)
          continue;
        const int d2 = di * di + dj * dj + dk * dk;
        if (d2 > R2) continue;
        const int ii = wrapc(S.i + di, N), jj = wrapc(S.j + dj, N), kk = wrapc(S.k + dk, N);
        const int64_t cell = B.off + ((int64_t)ii * N + jj) * N + kk;
        if (q == 0) {
          const double tout = 0.5 * dts;
          cube[cidx(0, 0, 0)] = tout;
          if (a.coldens) {
            a.coldens[cell] = tout / a.sigma0;
          } else {
            double dG;
            if (bits_of(tout) <= bits_of(a.tau_lim))
              dG = nd * (tab_eval(a.tab.h, a.tab, 0.0) * (0.5 * B.thin_fac));
            else
              dG = nd * ((tab_eval(a.tab.g, a.tab, 0.0) - tab_eval(a.tab.g, a.tab, tout)) *
                         B.inv_cell3 * a.invn[cell]);
            if (dG != 0.0) atomicAdd(&a.gamma[cell], dG);
          }
          continue;
        }
        const int adi = abs(di), adj = abs(dj), adk = abs(dk);
        const int m = max(adi, max(adj, adk));
        int D[3] = {di, dj, dk};
        int ax, x1, x2;
        if (adk == m) { ax = 2; x1 = 0; x2 = 1; }
        else if (adj == m) { ax = 1; x1 = 0; x2 = 2; }
        else { ax = 0; x1 = 1; x2 = 2; }
        const int p1 = D[x1], p2 = D[x2];
        const int ap1 = abs(p1), ap2 = abs(p2);
        const GeoEntry* ge = &a.geo[geo_index(m, min(ap1, ap2), max(ap1, ap2))];
        const double w1 = __ldg(&ge->w1), w4 = __ldg(&ge->w4), ds = __ldg(&ge->ds);
        const double w2 = ap1 <= ap2 ? __ldg(&ge->wa) : __ldg(&ge->wb);
        const double w3 = ap1 <= ap2 ? __ldg(&ge->wb) : __ldg(&ge->wa);
        double tin;
        if (m == 1) {
          tin = (0.5 * dts) * ds;
        } else {
          int e1[3] = {di, dj, dk};
          e1[ax] -= sgn_i(D[ax]);
          int e2[3] = {e1[0], e1[1], e1[2]};
          e2[x1] -= sgn_i(p1);
          int e3[3] = {e1[0], e1[1], e1[2]};
          e3[x2] -= sgn_i(p2);
          int e4[3] = {e2[0], e2[1], e2[2]};
          e4[x2] -= sgn_i(p2);
          const double c1 = cube[cidx(e1[0], e1[1], e1[2])];
          const double c2 = cube[cidx(e2[0], e2[1], e2[2])];
          const double c3 = cube[cidx(e3[0], e3[1], e3[2])];
          const double c4 = cube[cidx(e4[0], e4[1], e4[2])];
          tin = fma(w4, c4, fma(w3, c3, fma(w2, c2, w1 * c1)));
        }
        const double dtp = __ldg(&a.dtau[cell]);
        const double tout = fma(dtp, ds, tin);
        cube[cidx(di, dj, dk)] = tout;
        if (a.coldens) {
          a.coldens[cell] = tout / a.sigma0;
        } else if (bits_of(tin) < a.tab.tau_max_bits) {
          const double dcell = dtp * ds;
          const double dG = cell_rate(a, nd, tin, tout, dcell, __ldg(&ge->invv) * B.inv_cell3,
                                      __ldg(&ge->thin) * B.thin_fac,
                                      bits_of(dcell) <= bits_of(a.tau_lim) ? 0.0 : __ldg(&a.invn[cell]));
          ++nrate;
          if (dG != 0.0) atomicAdd(&a.gamma[cell], dG);
        }
      }
      __syncthreads();  // shell q complete before shell q+1 reads it
    }
  }
}

cudaError_t launch_trace_shells(Grid& g, const TraceArgs& a, int block, int grid) {
  switch (block) {
    case 128: k_trace_shells<128><<<grid, 128, 0, g.stream>>>(a); break;
    case 256: k_trace_shells<256><<<grid, 256, 0, g.stream>>>(a); break;
    case 512: k_trace_shells<512><<<grid, 512, 0, g.stream>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

int shells_max_grid(int block) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaErrorInvalidValue;
  if (block == 128) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_shells<128>, 128, 0);
  if (block == 256) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_shells<256>, 256, 0);
  if (block == 512) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_shells<512>, 512, 0);
  if (e != cudaSuccess) return 0;
  return per * sms;
}

}  // namespace asora

extern "C" int rt_shell_enumerate(int q, int32_t* h_out) {
  if (q < 0 || q > 100000) return -1;
  const int cnt = q == 0 ? 1 : 4 * q * q + 2;
  if (h_out)
    for (int t = 0; t < cnt; ++t) asora::shell_cell(q, t, h_out[3 * t], h_out[3 * t + 1], h_out[3 * t + 2]);
  return cnt;
}
