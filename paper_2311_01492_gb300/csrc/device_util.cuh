// Device helpers shared by the trace and adjoint kernels.
#pragma once

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
// nd_thick = Ndot / alpha^3 and nd_thin = Ndot sigma0 / alpha^2 are per source
// and box; the geometry entry holds 1/(4 pi r^2 ds) and 1/(4 pi r^2) in cell units.
// Only the branch taken reads its geometry and 1/n_HI.
__device__ __forceinline__ double cell_rate(const TraceArgs& a, double nd_thick, double nd_thin,
                                            double tin, double tout, double dcell,
                                            const GeoEntry* ge, const double* invn) {
  if (bits_of(dcell) <= bits_of(a.tau_lim))
    return nd_thin * (tab_eval(a.tab.h, a.tab, tin) * __ldg(&ge->thin));
  const double dg = tab_eval(a.tab.g, a.tab, tin) - tab_eval(a.tab.g, a.tab, tout);
  return nd_thick * (dg * (__ldg(&ge->invv) * __ldg(invn)));
}

// Interpolated column (Eq. interp) with optical-depth-modulated weights
// (interpolation mode 1, after the C2Ray paper's App. A, to which Sec. 3.1
// refers for the weighting): each geometric weight times r_n = 1/max(c_n, tw0),
// the sum normalised by the modulated weights, summed in the same order as the
// geometric chain.  The batched kernels keep r_n beside c_n in shared memory
// (formed once, when the cell's column is written, instead of once per reader).
__device__ __forceinline__ double od_interp_r(double w1, double w2, double w3, double w4,
                                              double c1, double c2, double c3, double c4,
                                              double r1, double r2, double r3, double r4,
                                              double nz) {
  const double v1 = w1 * r1, v2 = w2 * r2, v3 = w3 * r3, v4 = w4 * r4;
  const double S = ((v1 + v2) + v3) + v4;
  return fma(v4, c4, fma(v3, c3, fma(v2, c2, fma(v1, c1, nz)))) / S;
}
__device__ __forceinline__ double od_recip(double c, double tw0) { return 1.0 / fmax(c, tw0); }
__device__ __forceinline__ double od_interp(double w1, double w2, double w3, double w4, double c1,
                                            double c2, double c3, double c4, double tw0,
                                            double nz) {
  return od_interp_r(w1, w2, w3, w4, c1, c2, c3, c4, od_recip(c1, tw0), od_recip(c2, tw0),
                     od_recip(c3, tw0), od_recip(c4, tw0), nz);
}

// Slope of the table at tau (derivative of the lookup): the chord slope c1
// of tau's segment, 0 at and beyond the table's upper bound; -exp(-tau) for
// exact grey opacity.
__device__ __forceinline__ double tab_slope(const double2* __restrict__ t, const TabDev& tb,
                                            double tau) {
  if (tb.kind == RT_TABLE_GREY_EXACT) return -exp(-tau);
  const uint64_t b = bits_of(tau);
  if (b >= tb.tau_max_bits) return 0.0;
  int seg = 0;
  if (b >= tb.tau_min_bits) {
    const int e = (int)(b >> 52) - 1023;
    const int m = (int)((b >> (52 - tb.B)) & (uint64_t)((1 << tb.B) - 1));
    seg = 1 + ((e + tb.E0) << tb.B) + m;
  }
  return __ldg(&t[seg]).y;
}

// Row tables of one quadrant layer in shared memory (one slot): the first flat
// index of rows 0..nrows (nrows+1 ints) followed by the row of every flat index
// (bytes; rows < 256 since h <= 254), the same layout as the precomputed blobs;
// a slot holds any layer of half-width <= h.
__host__ __device__ inline int row_slot_bytes(int h) {
  return (4 * (h + 2) + (h + 1) * (h + 1) + 15) & ~15;
}

// Shared memory of one group tracing a quadrant of a face with layer half-width
// capacity h: two layers of (h+1)^2 doubles in CTA mode, one (updated in place)
// in warp mode -- with optical-depth-modulated weights (od) followed by as many
// again for the reciprocals 1/max(tau_out, tau_w0) of the same slots -- then
// (16-byte aligned, for cp.async) two row-table slots: the current layer's and
// the next's.
__host__ __device__ inline size_t layer_bytes(int h, bool warp, bool od = false) {
  const size_t cap = (size_t)(h + 1) * (h + 1);
  return ((warp ? 1 : 2) * (od ? 2 : 1) * cap * sizeof(double) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t group_smem_bytes(int h, bool warp, bool od = false) {
  return layer_bytes(h, warp, od) + 2 * (size_t)row_slot_bytes(h);
}

// Shared memory of one warp tracing a whole face: the face layer, (2h+1)^2
// doubles updated in place (slot of transverse offset (t1, t2) at
// (t1+h)(2h+1) + t2+h; with od, then the reciprocals of the same slots), then
// two slots for the interior row tables (the current layer's and the next's).
// At least the single-quadrant warp layout of group_smem_bytes, which faces
// clipped by the window use instead.
__host__ __device__ inline size_t face_buf_bytes(int h, bool od = false) {
  return ((od ? 2 : 1) * (size_t)(2 * h + 1) * (2 * h + 1) * sizeof(double) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t whole_smem_bytes(int h, bool od = false) {
  const size_t w = face_buf_bytes(h, od) + 2 * (size_t)row_slot_bytes(h);
  const size_t q = group_smem_bytes(h, true, od);
  return w > q ? w : q;
}

// Asynchronous copy of a precomputed row-table blob (16-byte aligned, size a
// multiple of 16) into a shared-memory slot by the GS threads of a group; the
// copies complete at the next cp_async_wait_all of each issuing thread.
template <int GS>
__device__ __forceinline__ void stage_rows(const unsigned char* __restrict__ src, int bytes,
                                           unsigned char* dst, int gt) {
  for (int c = gt * 16; c < bytes; c += GS * 16) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst + c);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src + c) : "memory");
  }
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;\n" ::: "memory");
}

template <int GS>
__device__ __forceinline__ void group_sync() {
  if (GS == 32) __syncwarp(); else __syncthreads();
}

// Row tables of one quadrant layer built by a single warp (lane = 0..31), no
// synchronisation.  Rows a1 = 0..nrows-1 (|t1|); row a1 holds a2 = 0..min(w, lim2)
// with w = min(H, floor(sqrt(rem - a1^2))).  rowpre[a1] = first flat index of row
// a1, rowpre[nrows] = layer size, rowof[t] = row of flat index t.  Each lane
// handles a contiguous block of rows, so its rowof writes are one contiguous range.
__device__ __forceinline__ void quad_rows_warp(int rem, int H, int nrows, int lim2,
                                               int* __restrict__ rowpre,
                                               unsigned char* __restrict__ rowof, int lane) {
  const int per = (nrows + 31) >> 5;
  const int rb = lane * per, re = min(nrows, rb + per);
  int local = 0;
  for (int r = rb; r < re; ++r) local += min(min(H, isqrt_i(rem - r * r)), lim2) + 1;
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  int run = incl - local;
  for (int r = rb; r < re; ++r) {
    rowpre[r] = run;
    const int len = min(min(H, isqrt_i(rem - r * r)), lim2) + 1;
    for (int c = 0; c < len; ++c) rowof[run + c] = (unsigned char)r;
    run += len;
  }
  if (lane == 31) rowpre[nrows] = incl;
}

}  // namespace asora
