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
// and only the owning face (k before j before i) deposits the rate.  Each face
// splits again into four quadrants (see trace_face_item), so every source
// gives 24 independent work items, taken longest-first from a device queue by
// persistent groups: CTAs (k_trace_faces) for items with wide layers, single
// warps (k_trace_faces_warp) for the others.  A quadrant layer lives in shared
// memory ((H+1)^2 doubles; two buffers per CTA, one updated in place per
// warp), so a cell reads only the previous layer of its own item.  The faces of
// small sources are traced whole by one warp (k_trace_faces_whole_warp): a
// (2h+1)^2 layer updated in place, every cell of a face computed once.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "asora_internal.cuh"
#include "device_util.cuh"

namespace asora {

// ----------------------------------------------------------- face kernels
// block codes: 128/256 CTA mode, 32 warp mode, 4 whole-face warp mode
size_t faces_smem_bytes(int hcap, int block, bool od) {
  return block == 4 ? whole_smem_bytes(hcap, od) : group_smem_bytes(hcap, block == 32, od);
}

// Trace one (source, face, quadrant) item with a group of GS threads (gt =
// thread index in the group).  Within a face, a cell's interpolants never
// cross the lines t1 = 0 or t2 = 0 towards the other side, so each quadrant
// (sign of t1, sign of t2, the lines included) depends only on itself; the
// lines are traced by both neighbouring quadrants and owned by the + side.
// Layers m = 1..Lmax; every cell reads only layer m-1.
//
// CTA mode (GS > 32) keeps layer m-1 and layer m in two buffers.  Warp mode
// (GS == 32) keeps one buffer with a fixed row stride and updates it in place:
// the cells are taken in descending flat order, 32 at a time, and every lane
// reads its interpolants before any lane writes.  A cell reads only slots
// (b <= a1, e <= a2), whose flat index in the current layer is not above its
// own, so each such slot is rewritten in the same round (after the reads) or in
// a later round -- never before it is read.
//
// Row tables: for an item whose window does not clip any layer, the tables of
// layer m+1 are copied (cp.async) from the precomputed blobs of its R^2 limit
// while layer m is traced; otherwise warp 0 builds them during layer m.
template <int GS, bool COLDENS, bool OD>
__device__ __forceinline__ void trace_face_item(const TraceArgs& a, const int item, const int gt,
                                                unsigned char* __restrict__ sm, const int h,
                                                unsigned& nrate) {
  const int cap = (h + 1) * (h + 1);
  double* buf0 = reinterpret_cast<double*>(sm);
  double* buf1 = GS == 32 ? buf0 : buf0 + cap;
  const int roff = (GS == 32 ? 1 : 2) * cap;  // OD: 1/max(tau_out, tau_w0) of slot i at i + roff
  const int TS = row_slot_bytes(h);
  unsigned char* tab2 = sm + layer_bytes(h, GS == 32, OD);  // [2][TS], 16-byte aligned
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
  const int64_t scell = B.off + ((int64_t)S.i * N + S.j) * N + S.k;
  const double dts = a.dtau[scell];

  if (f == 4 && quad == 0 && gt == 0) {  // the source cell (q = 0), once per source
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
      ++nrate;
      if (dG != 0.0) atomicAdd(&a.gamma[scell], dG);
    }
  }

  // transverse axes (t1, t2) in increasing axis order, and the field layouts:
  //   z faces read dtauT (k,i,j): index = k N^2 + i N + j  (t1 = i, t2 = j)
  //   y faces read dtau  (i,j,k): index = i N^2 + j N + k  (t1 = i, t2 = k)
  //   x faces read dtau  (i,j,k): index = i N^2 + j N + k  (t1 = j, t2 = k)
  // 32-bit offsets within the box (the batched schedule requires n^3 < 2^31)
  const int NN = N * N;
  const int c1 = d == 0 ? S.j : S.i;           // source coordinate along t1
  const int c2 = d == 2 ? S.j : S.k;           // source coordinate along t2
  const int cd = d == 0 ? S.i : (d == 1 ? S.j : S.k);
  const int m1 = d == 1 ? NN : N;              // stride of t1
  const int md = d == 1 ? N : NN;              // stride of the layer axis
  const double* __restrict__ fld = (d == 2 ? a.dtauT : a.dtau) + B.off;

  double* prev = buf0;
  double* cur = buf1;
  int Hp = 0;
  const bool exit_ok = !COLDENS && a.early_exit;
  int head_done = 0;  // warp mode: top cells of this layer traced in the previous layer's last round
  // precomputed row tables of this item's R^2 limit, if its window clips no layer:
  // blob of layer m at a.rtab + toff[m], toff[m+1] - toff[m] bytes
  const int* toff = nullptr;
  if (R2 <= a.rtab_max_r2) {
    const int sl = a.rtab_slot[R2];
    if (sl >= 0 && a.rtab_hcap[sl] <= min(lim1, lim2)) toff = a.rtab_off + a.rtab_first[sl] - 1;
  }
  // row tables of layer 1 (slot 1); layer m+1's (slot (m+1)&1) during layer m
  if (Lmax >= 1) {
    const int H1 = min(1, isqrt_i(R2 - 1));
    if (H1 <= h) {
      if (toff) {
        stage_rows<GS>(a.rtab + toff[1], toff[2] - toff[1], tab2 + TS, gt);
        cp_async_wait_all();
      } else if (wid == 0) {
        const int nr = min(H1, lim1) + 1;
        int* pre = reinterpret_cast<int*>(tab2 + TS);
        quad_rows_warp(R2 - 1, H1, nr, lim2, pre, reinterpret_cast<unsigned char*>(pre + nr + 1),
                       lane);
      }
    }
  }
  // Warp mode, layers m >= 2 without the early exit: one cell of a layer (params
  // L) per lane, all reads before the warp sync, the write after it.
  struct LayerP {
    int m, Hp, lc, lay, gbase;
    const GeoRow* grow;
    const int* rowpre;
    const unsigned char* rowof;
  };
  auto warp_cell = [&](const LayerP& L, const int t, const bool act) {
    const int a1 = L.rowof[t];
    const int a2 = t - L.rowpre[a1];
    const int x1 = wrapc(c1 + q1 * a1, N), x2 = wrapc(c2 + q2 * a2, N);
    const int gidx = L.lay + x1 * m1 + x2;
    const double dtp = __ldg(&fld[gidx]);
    const GeoRow* gr = L.grow + a1 * (L.m + 1) + a2;
    const double2 wv0 = __ldg(reinterpret_cast<const double2*>(gr));      // w1, w2
    const double2 wv1 = __ldg(reinterpret_cast<const double2*>(gr) + 1);  // w3, w4
    const double ds = __ldg(&gr->ds);
    const int Wh = h + 1;
    const int b1 = min(a1, L.Hp), b2 = min(a1 - (a1 > 0), L.Hp);
    const int e1 = min(a2, L.Hp), e2 = min(a2 - (a2 > 0), L.Hp);
    const int i1 = b1 * Wh + e1, i2 = b2 * Wh + e1, i3 = b1 * Wh + e2, i4 = b2 * Wh + e2;
    double tin;
    if (OD)
      tin = od_interp_r(wv0.x, wv0.y, wv1.x, wv1.y, prev[i1], prev[i2], prev[i3], prev[i4],
                        prev[i1 + roff], prev[i2 + roff], prev[i3 + roff], prev[i4 + roff],
                        a.neg_zero);
    else
      tin = fma(wv1.y, prev[i4], fma(wv1.x, prev[i3], fma(wv0.y, prev[i2],
                                                         fma(wv0.x, prev[i1], a.neg_zero))));
    const double tout = fma(dtp, ds, tin);
    __syncwarp();  // every lane has read its interpolants before any lane writes
    if (!act) return;
    cur[a1 * Wh + a2] = tout;
    if (OD) cur[a1 * Wh + a2 + roff] = od_recip(tout, a.tau_w0);
    const bool own = ((d == 2) || (d == 1 ? a2 < L.m : (a1 < L.m && a2 < L.m))) &&
                     (a1 > 0 || q1 > 0) && (a2 > 0 || q2 > 0);
    if (!own) return;
    if (COLDENS || bits_of(tin) < a.tab.tau_max_bits) {
      const int64_t cell = B.off + (d == 2 ? (x1 * N + x2) * N + L.lc : gidx);
      if (COLDENS) {
        a.coldens[cell] = tout / a.sigma0;
      } else {
        const GeoEntry* ge = &a.geo[L.gbase + ((max(a1, a2) * (max(a1, a2) + 1)) >> 1) + min(a1, a2)];
        const double dcell = dtp * ds;
        const double dG = cell_rate(a, nd * B.inv_cell3, nd * B.thin_fac, tin, tout, dcell, ge,
                                    &a.invn[cell]);
        ++nrate;
        if (dG != 0.0) atomicAdd(&a.gamma[cell], dG);
      }
    }
  };
  // The cells of layer m not traced yet (all but its hd top ones), 32 per round in
  // descending flat order.  A last round with k < 32 cells left gives its other
  // lanes the top cells of layer m+1 when that is safe: those read layer m only in
  // rows above the rows the k cells write (and write only rows above those the k
  // cells read), and layer m+1's row table is in shared memory -- so they read
  // exactly what they would read after layer m, and the partly filled rounds of
  // the two layers become one.
  auto warp_layer = [&](const int m, const int H, const int total, const int hd, const int lc,
                        const int lay, const GeoRow* grow, const int gbase, const int* rowpre,
                        const unsigned char* rowof, const int Hn) {
    const LayerP Lc{m, Hp, lc, lay, gbase, grow, rowpre, rowof};
    int t0 = total - 1 - hd;
    for (; t0 >= 31; t0 -= 32) warp_cell(Lc, t0 - lane, true);
    if (t0 < 0) return;
    const int k = t0 + 1;  // cells left in layer m: flat indices 0..k-1
    if (toff && m < Lmax && Hn <= h && m + 1 <= a.geo_mmax) {
      cp_async_wait_all();  // layer m+1's row table (staged at the start of layer m)
      __syncwarp();
      const int nrn = min(Hn, lim1) + 1;
      const int* pren = reinterpret_cast<const int*>(tab2 + ((m + 1) & 1) * TS);
      const unsigned char* rown = reinterpret_cast<const unsigned char*>(pren + nrn + 1);
      const int totn = pren[nrn];
      const int head = min(32 - k, totn);
      // rows: the k cells write (and read) rows <= rowof[k-1]; the head cells read
      // rows >= min(rown[totn-head] - 1, H) and write rows >= rown[totn-head]
      if (head > 0 && head < totn && min((int)rown[totn - head] - 1, H) > (int)rowof[k - 1]) {
        const int lcn = wrapc(cd + sg * (m + 1), N);
        const LayerP Ln{m + 1, H, lcn, lcn * md, (int)geo_index(m + 1, 0, 0),
                        a.georow + georow_index(m + 1, 0, 0), pren, rown};
        const bool mine = lane < k;
        const LayerP L{mine ? Lc.m : Ln.m, mine ? Lc.Hp : Ln.Hp, mine ? Lc.lc : Ln.lc,
                       mine ? Lc.lay : Ln.lay, mine ? Lc.gbase : Ln.gbase,
                       mine ? Lc.grow : Ln.grow, mine ? Lc.rowpre : Ln.rowpre,
                       mine ? Lc.rowof : Ln.rowof};
        const int t = mine ? k - 1 - lane : totn - 1 - (lane - k);
        warp_cell(L, max(t, 0), mine || lane - k < head);
        head_done = head;
        return;
      }
    }
    warp_cell(Lc, max(t0 - lane, 0), t0 - lane >= 0);
  };
  group_sync<GS>();
  for (int m = 1; m <= Lmax; ++m) {
    const int rem = R2 - m * m;
    const int H = min(m, isqrt_i(rem));
    if (H > h || m > a.geo_mmax) {
      if (gt == 0) atomicOr(a.err, H > h ? ERR_LAYER_CAP : ERR_GEO);
      break;
    }
    const int nrows = min(H, lim1) + 1;
    const int* rowpre = reinterpret_cast<const int*>(tab2 + (m & 1) * TS);
    const unsigned char* rowof = reinterpret_cast<const unsigned char*>(rowpre + nrows + 1);
    const int total = rowpre[nrows];
    int Hn = 0;  // half-width of the next layer
    if (m < Lmax) {
      Hn = min(m + 1, isqrt_i(R2 - (m + 1) * (m + 1)));
      if (toff && Hn <= h)
        stage_rows<GS>(a.rtab + toff[m + 1], toff[m + 2] - toff[m + 1], tab2 + ((m + 1) & 1) * TS, gt);
    }
    const int W = GS == 32 ? h + 1 : H + 1, Wp = GS == 32 ? h + 1 : Hp + 1;
    const int lc = wrapc(cd + sg * m, N);
    const int lay = lc * md;
    const GeoRow* __restrict__ grow = a.georow + georow_index(m, 0, 0);
    const int gbase = (int)geo_index(m, 0, 0);
    bool opaque = true;  // every cell of this thread has tau_out >= the exit bound
    // Layer 1 takes its column from the source cell alone.  It runs as its own
    // instantiation of the cell loop: a branch on m inside the loop becomes a
    // predicated FP64 product in every round of every layer, and an FP64
    // instruction whose lanes are all predicated off still takes its full turn
    // on the FP64 pipe.
    const int hd = head_done;
    head_done = 0;
    auto cells = [&](auto first) {
      constexpr bool FIRST = decltype(first)::value;
      if constexpr (GS == 32 && !FIRST) {
        if (!exit_ok) {
          warp_layer(m, H, total, hd, lc, lay, grow, gbase, rowpre, rowof, Hn);
          return;
        }
      }
      for (int t0 = GS == 32 ? total - 1 - hd : gt; GS == 32 ? t0 >= 0 : t0 < total;
           t0 += GS == 32 ? -32 : GS) {
        // warp mode: lanes take t0, t0-1, ..., t0-31; lanes below 0 recompute cell 0
        // and write nothing
        const int t = GS == 32 ? max(t0 - lane, 0) : t0;
        const int a1 = rowof[t];
        const int a2 = t - rowpre[a1];
        const int x1 = wrapc(c1 + q1 * a1, N), x2 = wrapc(c2 + q2 * a2, N);
        const int gidx = lay + x1 * m1 + x2;
        const double dtp = __ldg(&fld[gidx]);
        const GeoRow* gr = grow + a1 * (m + 1) + a2;
        const double2 wv0 = __ldg(reinterpret_cast<const double2*>(gr));      // w1, w2
        const double2 wv1 = __ldg(reinterpret_cast<const double2*>(gr) + 1);  // w3, w4
        const double ds = __ldg(&gr->ds);
        double tin;
        if constexpr (FIRST) {
          tin = (0.5 * dts) * ds;
        } else {
          const double w1 = wv0.x, w2 = wv0.y, w3 = wv1.x, w4 = wv1.y;
          const int b1 = min(a1, Hp), b2 = min(a1 - (a1 > 0), Hp);
          const int e1 = min(a2, Hp), e2 = min(a2 - (a2 > 0), Hp);
          const int i1 = b1 * Wp + e1, i2 = b2 * Wp + e1, i3 = b1 * Wp + e2, i4 = b2 * Wp + e2;
          const double v1 = prev[i1];
          const double v2 = prev[i2];
          const double v3 = prev[i3];
          const double v4 = prev[i4];
          // w1*v1 as fma(w1, v1, -0.0): the same value for every input (the sum of the
          // exact product and -0 rounds like the product alone, and +0 + -0 = +0), on
          // GB300 issued as a DFMA, which retires at least as fast as a DMUL
          if (OD)
            tin = od_interp_r(w1, w2, w3, w4, v1, v2, v3, v4, prev[i1 + roff], prev[i2 + roff],
                              prev[i3 + roff], prev[i4 + roff], a.neg_zero);
          else
            tin = fma(w4, v4, fma(w3, v3, fma(w2, v2, fma(w1, v1, a.neg_zero))));
        }
        const double tout = fma(dtp, ds, tin);
        if (GS == 32) {
          __syncwarp();  // every lane has read layer m-1 before any lane writes
          if (t0 - lane < 0) continue;
        }
        cur[a1 * W + a2] = tout;
        if (OD) cur[a1 * W + a2 + roff] = od_recip(tout, a.tau_w0);
        opaque = opaque && bits_of(tout) >= a.exit_bits;
        const bool own = ((d == 2) || (d == 1 ? a2 < m : (a1 < m && a2 < m))) &&
                         (a1 > 0 || q1 > 0) && (a2 > 0 || q2 > 0);
        if (!own) continue;
        if (COLDENS || bits_of(tin) < a.tab.tau_max_bits) {
          // C-order index of the cell (the z faces gathered from the rotated copy)
          const int64_t cell = B.off + (d == 2 ? (x1 * N + x2) * N + lc : gidx);
          if (COLDENS) {
            a.coldens[cell] = tout / a.sigma0;
          } else {
            const GeoEntry* ge = &a.geo[gbase + ((max(a1, a2) * (max(a1, a2) + 1)) >> 1) + min(a1, a2)];
            const double dcell = dtp * ds;
            const double dG = cell_rate(a, nd * B.inv_cell3, nd * B.thin_fac, tin, tout, dcell, ge,
                                        &a.invn[cell]);
            ++nrate;
            if (dG != 0.0) atomicAdd(&a.gamma[cell], dG);
          }
        }
      }
    };
    if (m == 1) cells(std::true_type());
    else cells(std::false_type());
    if (m < Lmax && Hn <= h) {  // row tables of the next layer
      if (toff) {
        cp_async_wait_all();
      } else if (wid == 0) {
        const int nr = min(Hn, lim1) + 1;
        int* pre = reinterpret_cast<int*>(tab2 + ((m + 1) & 1) * TS);
        quad_rows_warp(R2 - (m + 1) * (m + 1), Hn, nr, lim2, pre,
                       reinterpret_cast<unsigned char*>(pre + nr + 1), lane);
      }
    }
    if (exit_ok) {
      // Exact early exit: if every cell of this layer has tau_out >= 2^E1 (1 + 2^-40),
      // every later tau_in (a convex combination plus non-negative increments,
      // rounding covered by the margin) is >= 2^E1 and all later rates are 0.
      bool all_opaque;
      if (GS == 32) {
        __syncwarp();
        all_opaque = __all_sync(0xffffffffu, opaque);
      } else {
        all_opaque = __syncthreads_and(opaque) != 0;
      }
      if (all_opaque) break;
    } else {
      group_sync<GS>();
    }
    double* tmp = prev;
    prev = cur;
    cur = tmp;
    Hp = H;
  }
}

// The four quadrants of a clipped face one after another, kept out of line so
// that it does not weigh on the registers of the whole-face loop.
template <int GS, bool COLDENS, bool OD>
__device__ __noinline__ void trace_face_by_quadrants(const TraceArgs& a, const int item,
                                                     const int gt, unsigned char* sm, const int h,
                                                     unsigned& nrate) {
  for (int k = 0; k < 4; ++k) {
    trace_face_item<GS, COLDENS, OD>(a, (item & ~3) | k, gt, sm, h, nrate);
    group_sync<GS>();
  }
}

// Cells of layer m of an unclipped face, as one list in the order the in-place
// update needs (j ascending):
//   E row: |t1| = m    (2 + 4 LE entries: (+-m, 0), then (+-m, +-a2), a2 = 1..LE)
//   E col: |t2| = m, |t1| < m   (2 + 4 min(LE, m-1) entries)
//   I:     1 <= |t1|, |t2| <= m-1, the four sign images of each interior position
//          of the quadrant, positions in descending row-table order
//   A:     the axes, levels a = LA..1 descending, images (0,+a) (0,-a) (+a,0) (-a,0),
//          then (0, 0)
// with LE = min(m, isqrt(rem - m^2)) (E exists only if the layer reaches |t| = m)
// and LA = min(H, m-1).  cls: which weights can be non-zero.
enum { CLS_EROW = 0, CLS_ECOL = 1, CLS_I = 2, CLS_AT1 = 3, CLS_AT2 = 4 };

__device__ __forceinline__ void face_cell(const int j, const int m, const int nEr, const int nE,
                                          const int nI, const int LA,
                                          const int* __restrict__ rowpre,
                                          const unsigned char* __restrict__ rowof, int& t1,
                                          int& t2, int& cls) {
  if (j < nEr) {
    cls = CLS_EROW;
    const int u = j - 2, a2 = 1 + (u >> 2), k = u & 3;
    t1 = (j < 2 ? j : k) & 1 ? -m : m;
    t2 = j < 2 ? 0 : ((k & 2) ? -a2 : a2);
  } else if (j < nE) {
    cls = CLS_ECOL;
    const int v = j - nEr, u = v - 2, a1 = 1 + (u >> 2), k = u & 3;
    t1 = v < 2 ? 0 : ((k & 1) ? -a1 : a1);
    t2 = (v < 2 ? v : (k >> 1)) & 1 ? -m : m;
  } else if (j < nE + 4 * nI) {
    cls = CLS_I;
    const int u = j - nE, p = nI - 1 - (u >> 2), k = u & 3;
    const int r = rowof[p];
    const int a1 = r + 1, a2 = p - rowpre[r] + 1;
    t1 = (k & 1) ? -a1 : a1;
    t2 = (k & 2) ? -a2 : a2;
  } else {
    const int u = j - nE - 4 * nI, lvl = LA - (u >> 2), k = u & 3;
    const bool on_t2 = k < 2 && u < 4 * LA;  // t1 = 0 and t2 != 0
    cls = on_t2 ? CLS_AT1 : CLS_AT2;
    const int sgn = (k & 1) ? -lvl : lvl;
    t1 = on_t2 || u >= 4 * LA ? 0 : sgn;
    t2 = on_t2 ? sgn : 0;
  }
}

// Trace one face of one source (item = its quadrant-0 item) with a group of GS
// threads: a CTA (GS > 32) or one warp (GS == 32).  The face layer lives in one
// buffer, updated in place; the cells of layer m are taken from the list of
// face_cell, GS at a time, and each round reads all its interpolants before any
// thread writes (a barrier, or a warp sync).  A cell's non-zero-weight
// interpolants are cells of layer m-1 that come at or after it in the list
// (I positions in descending row-table order read positions not above their
// own; the axes read only the axes, which come last, inward; the E cells read
// |t| = m-1), so no slot is rewritten before it is read.  Weights of zero may
// read any slot: every slot holds a finite value (zeroed at kernel start).
// Rounds whose cells all lie on an axis or on the face's rim have two non-zero
// weights per cell and take the two-term form, which rounds exactly like the
// full chain (the zero terms add exactly +0).  Faces whose layers the window
// clips are traced quadrant by quadrant (trace_face_item) instead.
template <int GS, bool COLDENS, bool OD>
__device__ __forceinline__ void trace_face_whole(const TraceArgs& a, const int item, const int gt,
                                                 unsigned char* __restrict__ sm, const int h,
                                                 unsigned& nrate) {
  const int s = item >> 5, f = (item >> 2) & 7;
  const SrcDev S = a.src[s];
  const BoxDev B = a.boxes[S.box];
  const int R2 = a.r2lim[s];
  // interior row tables of this limit (blob of layer m at itab + toff[m]), used
  // when no window clips the face's layers
  const int* toff = nullptr;
  if (R2 <= a.rtab_max_r2 && a.itab) {
    const int sl = a.rtab_slot[R2];
    if (sl >= 0 && a.rtab_hcap[sl] <= min(B.whi, -B.wlo)) toff = a.itab_off + a.rtab_first[sl] - 1;
  }
  if (!toff) {
    trace_face_by_quadrants<GS, COLDENS, OD>(a, item & ~3, gt, sm, h, nrate);
    return;
  }
  const int N = B.n;
  const double nd = a.ndot[s];
  const int d = f >> 1;
  const int sg = (f & 1) ? -1 : 1;
  int Lmax = sg > 0 ? B.whi : -B.wlo;
  Lmax = min(Lmax, isqrt_i(R2));
  const int64_t scell = B.off + ((int64_t)S.i * N + S.j) * N + S.k;
  const double dts = a.dtau[scell];

  if (f == 4 && gt == 0) {  // the source cell (q = 0), once per source
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
      ++nrate;
      if (dG != 0.0) atomicAdd(&a.gamma[scell], dG);
    }
  }

  // axes and layouts as in trace_face_item
  const int NN = N * N;
  const int c1 = d == 0 ? S.j : S.i;
  const int c2 = d == 2 ? S.j : S.k;
  const int cd = d == 0 ? S.i : (d == 1 ? S.j : S.k);
  const int m1 = d == 1 ? NN : N;
  const int md = d == 1 ? N : NN;
  const double* __restrict__ fld = (d == 2 ? a.dtauT : a.dtau) + B.off;

  const int W = 2 * h + 1;
  double* ctr = reinterpret_cast<double*>(sm) + h * W + h;  // slot of (t1, t2): ctr[t1 W + t2]
  const int roff = W * W;  // OD: 1/max(tau_out, tau_w0) of slot o at o + roff
  const int TS = row_slot_bytes(h);
  unsigned char* tab2 = sm + face_buf_bytes(h, OD);  // [2][TS], 16-byte aligned
  const bool exit_ok = !COLDENS && a.early_exit;
  const double half_dts = 0.5 * dts;
  // interior tables of layer 1 (slot 1); layer m+1's (slot (m+1)&1) during layer m
  if (Lmax >= 1 && min(1, isqrt_i(R2 - 1)) <= h) {
    stage_rows<GS>(a.itab + toff[1], toff[2] - toff[1], tab2 + TS, gt);
    cp_async_wait_all();
  }
  group_sync<GS>();
  for (int m = 1; m <= Lmax; ++m) {
    const int rem = R2 - m * m;
    const int H = min(m, isqrt_i(rem));
    if (H > h || m > a.geo_mmax) {
      if (gt == 0) atomicOr(a.err, H > h ? ERR_LAYER_CAP : ERR_GEO);
      break;
    }
    int Hn = 0;
    if (m < Lmax) {
      Hn = min(m + 1, isqrt_i(R2 - (m + 1) * (m + 1)));
      if (Hn <= h)
        stage_rows<GS>(a.itab + toff[m + 1], toff[m + 2] - toff[m + 1], tab2 + ((m + 1) & 1) * TS,
                       gt);
    }
    const int LA = min(H, m - 1);
    const int* rowpre = reinterpret_cast<const int*>(tab2 + (m & 1) * TS);
    const unsigned char* rowof = reinterpret_cast<const unsigned char*>(rowpre + LA + 1);
    const int nI = rowpre[LA];
    int nEr = 0, nE = 0;
    if (H == m) {
      const int LE = min(m, isqrt_i(rem - m * m));
      nEr = 2 + 4 * LE;
      nE = nEr + 2 + 4 * min(LE, m - 1);
    }
    const int total = nE + 4 * nI + 4 * LA + 1;
    const int lc = wrapc(cd + sg * m, N);
    const int lay = lc * md;
    const GeoRow* __restrict__ grow = a.georow + georow_index(m, 0, 0);
    const int gbase = (int)geo_index(m, 0, 0);
    bool opaque = true;  // every cell of this thread has tau_out >= the exit bound
    // layer 1 as its own instantiation of the cell loop, as in trace_face_item
    auto cells = [&](auto first) {
      constexpr bool FIRST = decltype(first)::value;
      for (int j0 = 0; j0 < total; j0 += GS) {
        const int j = j0 + gt;  // threads past the end recompute the last cell, write nothing
        int t1, t2, cls;
        face_cell(min(j, total - 1), m, nEr, nE, nI, LA, rowpre, rowof, t1, t2, cls);
        const int a1 = abs(t1), a2 = abs(t2);
        const int x1 = wrapc(c1 + t1, N), x2 = wrapc(c2 + t2, N);
        const int gidx = lay + x1 * m1 + x2;
        const double dtp = __ldg(&fld[gidx]);
        const GeoRow* gr = grow + a1 * (m + 1) + a2;
        const double2 wv0 = __ldg(reinterpret_cast<const double2*>(gr));      // w1, w2
        const double2 wv1 = __ldg(reinterpret_cast<const double2*>(gr) + 1);  // w3, w4
        const double ds = __ldg(&gr->ds);
        const int o1 = t1 * W + t2;              // slots of (t1, t2), (t1-s1, t2),
        const int o2 = o1 - sgn_i(t1) * W;       // (t1, t2-s2), (t1-s1, t2-s2)
        const int o3 = o1 - sgn_i(t2);
        const int o4 = o2 - sgn_i(t2);
        double tin;
        if constexpr (FIRST) {
          tin = half_dts * ds;
        } else if (OD) {
          tin = od_interp_r(wv0.x, wv0.y, wv1.x, wv1.y, ctr[o1], ctr[o2], ctr[o3], ctr[o4],
                            ctr[o1 + roff], ctr[o2 + roff], ctr[o3 + roff], ctr[o4 + roff],
                            a.neg_zero);
        } else if (__all_sync(0xffffffffu, cls != CLS_I)) {
          // rim row (w1 = w3 = 0), rim column (w1 = w2 = 0), axis t1 = 0 (w2 = w4 = 0),
          // axis t2 = 0 (w3 = w4 = 0)
          const bool er = cls == CLS_EROW, ec = cls == CLS_ECOL, rim = er || ec;
          const double wA = er ? wv0.y : (ec ? wv1.x : wv0.x);
          const int oA = er ? o2 : (ec ? o3 : o1);
          const double wB = rim ? wv1.y : (cls == CLS_AT1 ? wv1.x : wv0.y);
          const int oB = rim ? o4 : (cls == CLS_AT1 ? o3 : o2);
          tin = fma(wB, ctr[oB], fma(wA, ctr[oA], a.neg_zero));
        } else {
          // w1*c1 as fma(w1, c1, -0.0): the same value for every input (the sum of the
          // exact product and -0 rounds like the product alone, and +0 + -0 = +0), on
          // GB300 issued as a DFMA, which retires at least as fast as a DMUL
          tin = fma(wv1.y, ctr[o4], fma(wv1.x, ctr[o3], fma(wv0.y, ctr[o2],
                                                             fma(wv0.x, ctr[o1], a.neg_zero))));
        }
        const double tout = fma(dtp, ds, tin);
        group_sync<GS>();  // every thread has read layer m-1 before any thread writes
        if (j >= total) continue;
        ctr[o1] = tout;
        if (OD) ctr[o1 + roff] = od_recip(tout, a.tau_w0);
        opaque = opaque && bits_of(tout) >= a.exit_bits;
        const bool own = (d == 2) || (d == 1 ? a2 < m : (a1 < m && a2 < m));
        if (!own) continue;
        if (COLDENS || bits_of(tin) < a.tab.tau_max_bits) {
          // C-order index of the cell (the z faces gathered from the rotated copy)
          const int64_t cell = B.off + (d == 2 ? (x1 * N + x2) * N + lc : gidx);
          if (COLDENS) {
            a.coldens[cell] = tout / a.sigma0;
          } else {
            const GeoEntry* ge = &a.geo[gbase + ((max(a1, a2) * (max(a1, a2) + 1)) >> 1) + min(a1, a2)];
            const double dcell = dtp * ds;
            const double dG = cell_rate(a, nd * B.inv_cell3, nd * B.thin_fac, tin, tout, dcell, ge,
                                        &a.invn[cell]);
            ++nrate;
            if (dG != 0.0) atomicAdd(&a.gamma[cell], dG);
          }
        }
      }
    };
    if (m == 1) cells(std::true_type());
    else cells(std::false_type());
    if (m < Lmax && Hn <= h) cp_async_wait_all();
    if (exit_ok) {
      // exact early exit, as in trace_face_item
      bool all_opaque;
      if (GS == 32) {
        __syncwarp();
        all_opaque = __all_sync(0xffffffffu, opaque);
      } else {
        all_opaque = __syncthreads_and(opaque) != 0;
      }
      if (all_opaque) break;
    } else {
      group_sync<GS>();
    }
  }
}

__device__ __forceinline__ void flush_rate_count(const TraceArgs& a, unsigned nrate) {
  if (!a.rate_cells) return;
  for (int o = 16; o > 0; o >>= 1) nrate += __shfl_down_sync(0xffffffffu, nrate, o);
  if ((threadIdx.x & 31) == 0 && nrate) atomicAdd(a.rate_cells, (unsigned long long)nrate);
}

// CTA mode: the whole CTA traces one item at a time (large sources).  Nine
// 128-thread CTAs per SM (56 registers; the shared memory of nine fits) measured
// faster than eight at 64 or fewer at 72-80 registers: latency, not registers,
// limits this loop.
template <int BLOCK, bool COLDENS, bool OD>
__global__ void __launch_bounds__(BLOCK, 1152 / BLOCK) k_trace_faces(TraceArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  if (a.skip && *a.skip) return;
  const int cap = (a.hcap + 1) * (a.hcap + 1);
  double* buf = reinterpret_cast<double*>(smem_raw);
  for (int t = threadIdx.x; t < (OD ? 4 : 2) * cap; t += BLOCK) buf[t] = 0.0;
  unsigned nrate = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = a.item_begin + atomicAdd(a.queue, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= a.n_items) break;
    trace_face_item<BLOCK, COLDENS, OD>(a, a.items[it], threadIdx.x, smem_raw, a.hcap, nrate);
  }
  flush_rate_count(a, nrate);
}

// Warp mode: every warp traces its own items (small sources), with its own
// slice of shared memory and warp-level synchronisation only.
// The CTA holds 1..8 warps (blockDim.x / 32), chosen at launch so that the most
// warps stay resident for the shared memory one warp needs.
template <bool COLDENS, bool OD>
__global__ void __launch_bounds__(256, 4) k_trace_faces_warp(TraceArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.skip && *a.skip) return;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* my = smem_raw + (size_t)wid * group_smem_bytes(a.hcap, true, OD);
  const int cap = (a.hcap + 1) * (a.hcap + 1);
  double* buf = reinterpret_cast<double*>(my);
  for (int t = lane; t < (OD ? 2 : 1) * cap; t += 32) buf[t] = 0.0;  // one layer buffer per warp
  __syncwarp();
  unsigned nrate = 0;
  for (;;) {
    int it = 0;
    if (lane == 0) it = a.item_begin + atomicAdd(a.queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= a.n_items) break;
    trace_face_item<32, COLDENS, OD>(a, a.items[it], lane, my, a.hcap, nrate);
    __syncwarp();
  }
  flush_rate_count(a, nrate);
}

// Whole-face warp mode kernel: every warp traces whole faces (small sources);
// items are faces, face it being the quadrant-0 item items[4 it].  Up to 80
// registers (measured faster than 64, where the loop spills); shared memory
// bounds the warps per SM for these faces anyway.
template <bool COLDENS, bool OD>
__global__ void __launch_bounds__(256, 3) k_trace_faces_whole_warp(TraceArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  if (a.skip && *a.skip) return;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* my = smem_raw + (size_t)wid * whole_smem_bytes(a.hcap, OD);
  const int W = 2 * a.hcap + 1;
  double* buf = reinterpret_cast<double*>(my);
  for (int t = lane; t < (OD ? 2 : 1) * W * W; t += 32) buf[t] = 0.0;  // one face buffer per warp
  __syncwarp();
  unsigned nrate = 0;
  for (;;) {
    int it = 0;
    if (lane == 0) it = a.item_begin + atomicAdd(a.queue, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= a.n_items) break;
    trace_face_whole<32, COLDENS, OD>(a, a.items[4 * it], lane, my, a.hcap, nrate);
    __syncwarp();
  }
  flush_rate_count(a, nrate);
}

// Kernel variant for (block, warps per CTA, coldens): block 128/256 = CTA mode,
// 32 = warp mode and 4 = whole-face warp mode with wpb warps per CTA (1..8).  Null
// if not instantiated.
static const void* face_kernel(int block, int wpb, bool coldens, bool od) {
#define ASORA_PICK(K) (od ? (coldens ? (const void*)K<true, true> : (const void*)K<false, true>) \
                          : (coldens ? (const void*)K<true, false> : (const void*)K<false, false>))
  switch (block) {
    case 32:
      if (wpb < 1 || wpb > 8) return nullptr;
      return ASORA_PICK(k_trace_faces_warp);
    case 4:  // whole-face warp mode, wpb warps per CTA
      if (wpb < 1 || wpb > 8) return nullptr;
      return ASORA_PICK(k_trace_faces_whole_warp);
    case 128:
      return od ? (coldens ? (const void*)k_trace_faces<128, true, true>
                           : (const void*)k_trace_faces<128, false, true>)
                : (coldens ? (const void*)k_trace_faces<128, true, false>
                           : (const void*)k_trace_faces<128, false, false>);
    case 256:
      return od ? (coldens ? (const void*)k_trace_faces<256, true, true>
                           : (const void*)k_trace_faces<256, false, true>)
                : (coldens ? (const void*)k_trace_faces<256, true, false>
                           : (const void*)k_trace_faces<256, false, false>);
    default: return nullptr;
  }
#undef ASORA_PICK
}

cudaError_t launch_trace_faces(Grid& g, const TraceArgs& a, int block, int grid, size_t smem,
                               int wpb) {
  const bool cd = a.coldens != nullptr;
  const void* fn = face_kernel(block, wpb, cd, a.interp_mode == RT_INTERP_OPTICAL_DEPTH);
  if (!fn) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int threads = (block == 32 || block == 4) ? wpb * 32 : block;
  TraceArgs arg = a;
  void* params[] = {&arg};
  e = cudaLaunchKernel(fn, dim3(grid), dim3(threads), params, smem, g.stream);
  count_launch();
  return e;
}

int faces_max_grid(int block, size_t smem, int wpb, bool od) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = face_kernel(block, wpb, false, od);
  if (!fn) return 0;
  const int threads = (block == 32 || block == 4) ? wpb * 32 : block;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, threads, smem);
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

template <int BLOCK, bool OD>
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
      // Cells with max|Delta| = 1 (and the source cell) lie in shells q <= 3 only;
      // the later shells run an instantiation without those branches, which would
      // otherwise issue FP64 products with every lane predicated off.
      auto cells = [&](auto near) {
        constexpr bool NEAR = decltype(near)::value;
        for (int t = tid; t < cnt; t += BLOCK) {
          int di, dj, dk;
          shell_cell(q, t, di, dj, dk);
          if (di < B.wlo || di > B.whi || dj < B.wlo || dj > B.whi || dk < B.wlo || dk > B.whi)
            continue;
          const int d2 = di * di + dj * dj + dk * dk;
          if (d2 > R2) continue;
          const int ii = wrapc(S.i + di, N), jj = wrapc(S.j + dj, N), kk = wrapc(S.k + dk, N);
          const int64_t cell = B.off + ((int64_t)ii * N + jj) * N + kk;
          if (NEAR && q == 0) {
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
          if (NEAR && m == 1) {
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
            if (OD)
              tin = od_interp(w1, w2, w3, w4, c1, c2, c3, c4, a.tau_w0, a.neg_zero);
            else
              tin = fma(w4, c4, fma(w3, c3, fma(w2, c2, w1 * c1)));
          }
          const double dtp = __ldg(&a.dtau[cell]);
          const double tout = fma(dtp, ds, tin);
          cube[cidx(di, dj, dk)] = tout;
          if (a.coldens) {
            a.coldens[cell] = tout / a.sigma0;
          } else if (bits_of(tin) < a.tab.tau_max_bits) {
            const double dcell = dtp * ds;
            const double dG = cell_rate(a, nd * B.inv_cell3, nd * B.thin_fac, tin, tout, dcell, ge,
                                        &a.invn[cell]);
            ++nrate;
            if (dG != 0.0) atomicAdd(&a.gamma[cell], dG);
          }
        }
      };
      if (q <= 3) cells(std::true_type());
      else cells(std::false_type());
      __syncthreads();  // shell q complete before shell q+1 reads it
    }
  }
}

cudaError_t launch_trace_shells(Grid& g, const TraceArgs& a, int block, int grid) {
  const bool od = a.interp_mode == RT_INTERP_OPTICAL_DEPTH;
  switch (block) {
    case 128:
      if (od) k_trace_shells<128, true><<<grid, 128, 0, g.stream>>>(a);
      else k_trace_shells<128, false><<<grid, 128, 0, g.stream>>>(a);
      break;
    case 256:
      if (od) k_trace_shells<256, true><<<grid, 256, 0, g.stream>>>(a);
      else k_trace_shells<256, false><<<grid, 256, 0, g.stream>>>(a);
      break;
    case 512:
      if (od) k_trace_shells<512, true><<<grid, 512, 0, g.stream>>>(a);
      else k_trace_shells<512, false><<<grid, 512, 0, g.stream>>>(a);
      break;
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
  if (block == 128) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_shells<128, false>, 128, 0);
  if (block == 256) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_shells<256, false>, 256, 0);
  if (block == 512) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace_shells<512, false>, 512, 0);
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
