// Discrete adjoint of one LTS sweep (Sec. 2.6 with the Jacobi reading of the
// sweep), for a fixed integer schedule.  One reverse sweep, given the adjoint
// of the state after the sweep, runs in the reverse order of the forward:
//   k_adj_elem    phase B of every ready element: recompute reconstruction
//                 and predictor from the post-sweep state, reverse them, and
//                 scatter to the element and its stencil members' virtual data
//   k_adj_commit  moved nodes: the adjoint of their committed position moves
//                 to the new position of the sweep
//   k_adj_update  one-step FV update / memory variables (eqs. PDEfinal, Qm2)
//   k_adj_edges   swept edge surfaces: Rusanov ALE flux through Gauss points
//   k_adj_nodes   node solver NS_cs (eqs. eqnNScs, NodesVel, newVertex)
// The lists of the sweep (ready elements, moved nodes, active edges, touched
// elements) and the new node positions come from re-running the forward
// k_ready, k_nodes and k_edges on the sweep-start state, which they read
// where its snapshot holds it (they write only lists and scratch).  Scatters to
// other elements and nodes use atomics; the slots an element owns (its
// tables, its edges' traces) are written by one thread only.
#include <algorithm>
#include <cfloat>
#include <climits>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>

#include "aw_adjoint_elem.cuh"
#include "aw_internal.h"

namespace aw {

namespace {

using adj::Sz;

__device__ __forceinline__ void set_error(Counters* cnt, int code, int elem) {
  if (atomicCAS(&cnt->err_code, 0, code) == 0) cnt->err_elem = elem;
}

// Work space of one element's phase-B reverse (shared memory of its warp).
template <int M>
struct ElemWork {
  using S = Sz<M>;
  adj::ReconIn<M> in;
  adj::ReconTape<M> rt;
  adj::PredTape<M> pt;
  adj::PredTables<M> tab, tb;
  double wb[S::Mc][4];
  double Xb[6], Qb[4];
  double Xvb[S::MaxU][6], Qvb[S::MaxU][4];
  double mem_tau[S::MaxU], mem_dts[S::MaxU];
  int mem_j[S::MaxU];
  union Scratch {
    adj::PredWork<M> pw;
    adj::PredRev<M> pr;
    adj::ReconRev<M> rr;
  } sc;
};

// Phase B of one element, reversed: one block of kElemThreads threads per
// element (all four SM sub-partitions share its FP64 work), its recomputed
// forward data and adjoints in shared memory.
constexpr int kElemThreads = 128;

template <int M>
__global__ void __launch_bounds__(kElemThreads, 4) k_adj_elem(Tab T, Dev post, Dev live, Adj a, int initial) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc, Nt = S::Nt, NE = S::NE, MaxU = S::MaxU, NT = kElemThreads;
  extern __shared__ double smem_elem[];
  __shared__ double red[NT / 32];
  ElemWork<M>& W = *reinterpret_cast<ElemWork<M>*>(smem_elem);
  const adj::TeamBlock tm{(int)threadIdx.x, NT, red};
  const int lane = threadIdx.x;
  const int n = initial ? post.ne : live.cnt->n_ready;
  for (int pos = blockIdx.x; pos < n; pos += gridDim.x) {
    const int i = initial ? pos : live.ready_list[pos];
    // adjoints of the element's new tables (overwritten by this sweep, so
    // their adjoint restarts from zero before phase A).  Where they are all
    // zero the element's reverse contributes exact zeros: skip it.
    int nz = 0;
    {
      double* tr = a.trb + (size_t)i * 3 * Nt * Nt * 4;
      double* av = a.avb + (size_t)i * Nt * 4;
      double* vd = a.vdb + (size_t)i * 6 * Nt;
      for (int k = lane; k < 3 * Nt * Nt * 4; k += NT) {
        const double v = tr[k];
        (&W.tb.tr[0][0][0][0])[k] = v;
        nz |= v != 0.0;
        tr[k] = 0.0;
      }
      for (int k = lane; k < Nt * 4; k += NT) {
        const double v = av[k];
        (&W.tb.av[0][0])[k] = v;
        nz |= v != 0.0;
        av[k] = 0.0;
      }
      for (int k = lane; k < 6 * Nt; k += NT) {
        const double v = vd[k];
        (&W.tb.vd[0][0])[k] = v;
        nz |= v != 0.0;
        vd[k] = 0.0;
      }
    }
    if (!tm.any(nz)) continue;
    const long long ti = post.t[i];
    const int u0 = post.u_ptr[i], nU = post.u_ptr[i + 1] - u0;
    const double dts = (double)post.dt[i] * post.etick[i];
    const int nit = dts > 0.0 ? T.nit : 0;
    if (nU > MaxU || nit > adj::kMaxIt) {
      if (lane == 0) set_error(live.cnt, -7, i);
      continue;
    }
    if (lane < 6) W.in.X[lane] = post.X[6 * (size_t)i + lane];
    if (lane < 4) W.in.Q[lane] = post.Q[4 * (size_t)i + lane];
    if (lane == 0) W.in.nU = nU;
    for (int k = lane; k < kNSten * NE; k += NT) W.in.st[k / NE][k % NE] = post.sten[(size_t)i * kNSten * NE + k];
    for (int s = lane; s < kNSten; s += NT) W.in.ok[s] = post.sten_ok[(size_t)i * kNSten + s];
    for (int u = lane; u < nU; u += NT) {
      const int j = post.u_elem[u0 + u];
      W.mem_j[u] = j;
      const long long tj = post.t[j], dtj = post.dt[j];
      double* Xv = W.in.Xv[u];
      for (int k = 0; k < 6; ++k) Xv[k] = post.X[6 * (size_t)j + k];
      if (tj == ti || dtj == 0) {
        W.mem_tau[u] = -1.0;  // real data of the member
        W.mem_dts[u] = 0.0;
        for (int v = 0; v < 4; ++v) W.in.Qv[u][v] = post.Q[4 * (size_t)j + v];
      } else {
        const double tau = (double)(ti - tj) / (double)dtj;
        const double dtsj = (double)dtj * post.etick[j];
        W.mem_tau[u] = tau;
        W.mem_dts[u] = dtsj;
        const double* vd = post.vdisp + (size_t)j * 6 * Nt;
        for (int kc = 0; kc < 6; ++kc) {
          double acc = vd[kc * Nt + Nt - 1];
          for (int p = Nt - 2; p >= 0; --p) acc = acc * tau + vd[kc * Nt + p];
          Xv[kc] += dtsj * (acc * tau);
        }
        const double* av = post.avgc + (size_t)j * Nt * 4;
        for (int v = 0; v < 4; ++v) {
          double acc = av[(Nt - 1) * 4 + v];
          for (int p = Nt - 2; p >= 0; --p) acc = acc * tau + av[p * 4 + v];
          W.in.Qv[u][v] = acc;
        }
      }
      const double sx = post.u_shift[2 * (size_t)(u0 + u)], sy = post.u_shift[2 * (size_t)(u0 + u) + 1];
      for (int k = 0; k < 3; ++k) {
        Xv[2 * k] += sx;
        Xv[2 * k + 1] += sy;
      }
      for (int k = 0; k < 6; ++k) W.Xvb[u][k] = 0.0;
      for (int v = 0; v < 4; ++v) W.Qvb[u][v] = 0.0;
    }
    for (int k = lane; k < Mc * 4; k += NT) (&W.wb[0][0])[k] = 0.0;
    if (lane < 6) W.Xb[lane] = 0.0;
    if (lane < 4) W.Qb[lane] = 0.0;
    tm.sync();
    adj::recon_fwd<M>(T, W.in, W.rt, tm);
    if (W.rt.limited) {  // the positivity scaling is a kink of the map
      if (lane == 0) set_error(live.cnt, -7, i);
      tm.sync();
      continue;
    }
    adj::pred_fwd<M>(T, nit, W.rt.w, W.in.X, dts, W.pt, W.tab, W.sc.pw, tm);
    if (W.pt.bad) {
      if (lane == 0) set_error(live.cnt, -7, i);
      tm.sync();
      continue;
    }
    adj::pred_rev<M>(T, nit, dts, W.pt, W.tb, W.wb, W.Xb, W.sc.pr, tm);
    adj::recon_rev<M>(T, W.in, W.rt, W.wb, W.Xb, W.Qb, W.Xvb, W.Qvb, W.sc.rr, tm);
    for (int u = lane; u < nU; u += NT) {
      const int j = W.mem_j[u];
      for (int k = 0; k < 6; ++k) atomicAdd(&a.Xb[6 * (size_t)j + k], W.Xvb[u][k]);
      if (W.mem_tau[u] < 0.0) {
        for (int v = 0; v < 4; ++v) atomicAdd(&a.Qb[4 * (size_t)j + v], W.Qvb[u][v]);
      } else {
        const double tau = W.mem_tau[u], dtsj = W.mem_dts[u];
        double* vd = a.vdb + (size_t)j * 6 * Nt;
        for (int kc = 0; kc < 6; ++kc) {
          double tp = tau;
          for (int p = 0; p < Nt; ++p) {
            atomicAdd(&vd[kc * Nt + p], W.Xvb[u][kc] * dtsj * tp);
            tp *= tau;
          }
        }
        double* av = a.avb + (size_t)j * Nt * 4;
        double tp = 1.0;
        for (int p = 0; p < Nt; ++p) {
          for (int v = 0; v < 4; ++v) atomicAdd(&av[p * 4 + v], W.Qvb[u][v] * tp);
          tp *= tau;
        }
      }
    }
    if (lane < 6) atomicAdd(&a.Xb[6 * (size_t)i + lane], W.Xb[lane]);
    if (lane < 4) atomicAdd(&a.Qb[4 * (size_t)i + lane], W.Qb[lane]);
    tm.sync();
  }
}

__global__ void k_adj_commit(Dev d, Adj a) {
  const int n_moved = d.cnt->n_moved;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n_moved; q += gridDim.x * blockDim.x) {
    const int n = d.moved_list[q];
    a.nXnb[2 * n] = a.nXb[2 * n];
    a.nXnb[2 * n + 1] = a.nXb[2 * n + 1];
    a.nXb[2 * n] = 0.0;
    a.nXb[2 * n + 1] = 0.0;
  }
}

// FV update of a ready element: |T'| Q' = |T| Q - sum sign G + QM, QM' = 0,
// X' = new corners; a touched element that is not ready: QM' = QM - sum sign G
__global__ void k_adj_update(Dev live, Dev post, Adj a) {
  const int epoch = live.cnt->epoch;
  const int n = live.cnt->n_touched;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n; q += gridDim.x * blockDim.x) {
    const int i = live.touch_list[q];
    if (live.elem_ready[i] == epoch) {
      const double* Xn = post.X + 6 * (size_t)i;
      const double* Xo = live.X + 6 * (size_t)i;
      const double Anew = adj::tri_area(Xn), Aold = adj::tri_area(Xo);
      double nb[4], Anb = 0.0, Aob = 0.0;
      for (int v = 0; v < 4; ++v) {
        nb[v] = a.Qb[4 * (size_t)i + v] / Anew;
        Anb -= nb[v] * post.Q[4 * (size_t)i + v];
        Aob += nb[v] * live.Q[4 * (size_t)i + v];
      }
      for (int v = 0; v < 4; ++v) {
        a.Qb[4 * (size_t)i + v] = Aold * nb[v];
        a.QMb[4 * (size_t)i + v] = nb[v];
        a.gb[4 * (size_t)i + v] = nb[v];
      }
      double Xnb[6];
      for (int k = 0; k < 6; ++k) Xnb[k] = a.Xb[6 * (size_t)i + k];
      adj::tri_area_rev(Xn, Anb, Xnb);
      for (int k = 0; k < 3; ++k) {
        const int nd = live.tri[3 * (size_t)i + k];
        atomicAdd(&a.nXnb[2 * nd], Xnb[2 * k]);
        atomicAdd(&a.nXnb[2 * nd + 1], Xnb[2 * k + 1]);
      }
      double Xob[6] = {0, 0, 0, 0, 0, 0};
      adj::tri_area_rev(Xo, Aob, Xob);
      for (int k = 0; k < 6; ++k) a.Xb[6 * (size_t)i + k] = Xob[k];
    } else {
      for (int v = 0; v < 4; ++v) a.gb[4 * (size_t)i + v] = a.QMb[4 * (size_t)i + v];
    }
  }
}

// One lane per Gauss point: (M+1)^2 consecutive lanes per active edge,
// 32 / (M+1)^2 edges per warp; the corner adjoints are summed over the points
// by a shuffle tree within the edge's lanes, the trace adjoints of one Gauss
// row onto the row's first lane.
template <int M>
__global__ void __launch_bounds__(128) k_adj_edges(Tab T, Dev d, Adj a) {
  constexpr int Nt = M + 1, NP = Nt * Nt, EPW = 32 / NP;
  const int epoch = d.cnt->epoch;
  const int n_active = d.cnt->n_active;
  const int n_items = (n_active + EPW - 1) / EPW * 32;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n_items; base += stride) {
    const int item = base + threadIdx.x;
    const int lane = item & 31, slot = lane / NP, pt = lane % NP;
    const int q = (item >> 5) * EPW + slot;
    const bool valid = item < n_items && slot < EPW && q < n_active;
    double Pb[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
    double trLb[Nt][Nt][4], trRb[Nt][Nt][4], qgb[4] = {0, 0, 0, 0};
    int na = 0, nb_ = 0, gxl = -1, Ll = 0, lel = 0, Rl = -1, lrl = 0;
    bool trans = false;
    bool ma = false, mb = false;
    if (valid) {
      const int ed = d.active_list[q];
      na = d.edge_nodes[2 * ed];
      nb_ = d.edge_nodes[2 * ed + 1];
      ma = d.node_moved[na] == epoch;
      mb = d.node_moved[nb_] == epoch;
      {
        const int L = d.edge_elem[2 * ed], R = d.edge_elem[2 * ed + 1];
        const int le = d.edge_loc[2 * ed], lr = d.edge_loc[2 * ed + 1];
        const int le1 = le == 2 ? 0 : le + 1;
        const double sax = d.cshift[6 * (size_t)L + 2 * le], say = d.cshift[6 * (size_t)L + 2 * le + 1];
        const double sbx = d.cshift[6 * (size_t)L + 2 * le1], sby = d.cshift[6 * (size_t)L + 2 * le1 + 1];
        adj::EdgeIn<M> in;
        in.P[0][0] = d.nX[2 * na] + sax; in.P[0][1] = d.nX[2 * na + 1] + say; in.tk[0] = (double)d.nt[na];
        in.P[1][0] = d.nX[2 * nb_] + sbx; in.P[1][1] = d.nX[2 * nb_ + 1] + sby; in.tk[1] = (double)d.nt[nb_];
        if (mb) { in.P[2][0] = d.nXn[2 * nb_] + sbx; in.P[2][1] = d.nXn[2 * nb_ + 1] + sby; in.tk[2] = (double)d.ntn[nb_]; }
        else { in.P[2][0] = in.P[1][0]; in.P[2][1] = in.P[1][1]; in.tk[2] = in.tk[1]; }
        if (ma) { in.P[3][0] = d.nXn[2 * na] + sax; in.P[3][1] = d.nXn[2 * na + 1] + say; in.tk[3] = (double)d.ntn[na]; }
        else { in.P[3][0] = in.P[0][0]; in.P[3][1] = in.P[0][1]; in.tk[3] = in.tk[0]; }
        in.tsec = d.etick[L];
        in.tL = (double)d.t[L];
        in.dtL = (double)d.dt[L];
        const int gx = pt / Nt, gt = pt % Nt;
        const double* cL = d.trace + (((size_t)L * 3 + le) * Nt) * Nt * 4;
        for (int k = 0; k < Nt * 4; ++k) (&in.trL[gx][0][0])[k] = cL[gx * Nt * 4 + k];
        in.has_R = R >= 0;
        in.bc = d.edge_bc[ed];
        trans = R < 0 && in.bc == 1;
        for (int v = 0; v < 4; ++v) in.qg[v] = trans ? d.Q[4 * (size_t)L + v] : 0.0;
        if (R >= 0) {
          in.tR = (double)d.t[R];
          in.dtR = (double)d.dt[R];
          const double* cR = d.trace + (((size_t)R * 3 + lr) * Nt) * Nt * 4;
          const int gr = Nt - 1 - gx;
          for (int k = 0; k < Nt * 4; ++k) (&in.trR[gr][0][0])[k] = cR[gr * Nt * 4 + k];
        }
        double Gb[4];
        for (int v = 0; v < 4; ++v) Gb[v] = -a.gb[4 * (size_t)L + v] + (R >= 0 ? a.gb[4 * (size_t)R + v] : 0.0);
        for (int p = 0; p < Nt; ++p)
          for (int v = 0; v < 4; ++v) trLb[gx][p][v] = trRb[Nt - 1 - gx][p][v] = 0.0;
        // a zero flux adjoint contributes exact zeros
        if (Gb[0] != 0.0 || Gb[1] != 0.0 || Gb[2] != 0.0 || Gb[3] != 0.0)
          adj::edge_point_rev<M>(T, in, gx, gt, Gb, Pb, trLb, trRb, qgb);
        gxl = gx;
        Ll = L; lel = le; Rl = R; lrl = lr;
      }
    }
    // the Nt points of one Gauss row (gx) are consecutive lanes: sum their
    // trace adjoints onto the row's first lane, which owns the edge's slots
    // (each element edge belongs to one swept edge only)
#pragma unroll
    for (int k = 0; k < Nt * 4; ++k) {
      double l_ = gxl >= 0 ? (&trLb[gxl][0][0])[k] : 0.0, r_ = gxl >= 0 ? (&trRb[Nt - 1 - gxl][0][0])[k] : 0.0;
      double ls = l_, rs = r_;
#pragma unroll
      for (int o = 1; o < Nt; ++o) {
        const double lo = __shfl_down_sync(0xffffffffu, l_, o), ro = __shfl_down_sync(0xffffffffu, r_, o);
        ls += lo;
        rs += ro;
      }
      if (gxl >= 0 && pt % Nt == 0) {
        a.trb[(((size_t)Ll * 3 + lel) * Nt + gxl) * Nt * 4 + k] += ls;
        if (Rl >= 0) a.trb[(((size_t)Rl * 3 + lrl) * Nt + (Nt - 1 - gxl)) * Nt * 4 + k] += rs;
      }
    }
#pragma unroll
    for (int off = 1; off < NP; off <<= 1) {
      const bool in = pt + off < NP;
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const double o = __shfl_down_sync(0xffffffffu, Pb[k][c], off);
          if (in) Pb[k][c] += o;
        }
    }
    // transmissive outer state: the left element's sweep-start average
#pragma unroll
    for (int off = 1; off < NP; off <<= 1) {
      const bool in = pt + off < NP;
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double o = __shfl_down_sync(0xffffffffu, qgb[v], off);
        if (in) qgb[v] += o;
      }
    }
    if (valid && pt == 0 && trans)
      for (int v = 0; v < 4; ++v) atomicAdd(&a.Qb[4 * (size_t)Ll + v], qgb[v]);
    if (valid && pt == 0)
      for (int c = 0; c < 2; ++c) {
        atomicAdd(&a.nXb[2 * na + c], Pb[0][c] + (ma ? 0.0 : Pb[3][c]));
        atomicAdd(&a.nXb[2 * nb_ + c], Pb[1][c] + (mb ? 0.0 : Pb[2][c]));
        if (mb) atomicAdd(&a.nXnb[2 * nb_ + c], Pb[2][c]);
        if (ma) atomicAdd(&a.nXnb[2 * na + c], Pb[3][c]);
      }
  }
}

// Node solver reversed with 8 lanes per moved node, one Voronoi element per
// lane (strided): D = sum mu_j D_j / sum mu_j with mu_j = rho_j |T_j|.
__global__ void k_adj_nodes_grp(Tab T, Dev d, Adj a) {
  constexpr int GS = 8;
  const int Nt = T.Nt;
  const int n_items = d.cnt->n_moved * GS;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x; base < n_items; base += stride) {
    const int item = base + threadIdx.x;
    const int q = item / GS, lane = item % GS;
    const bool live = item < n_items;
    int n = 0, p0 = 0, p1 = 0, ty = 0;
    double Db[2] = {0.0, 0.0};
    long long tk0 = 0, tk1 = 0;
    if (live) {
      n = d.moved_list[q];
      Db[0] = a.nXnb[2 * n];
      Db[1] = a.nXnb[2 * n + 1];
      if (lane == 0) {
        a.nXb[2 * n] += Db[0];
        a.nXb[2 * n + 1] += Db[1];
      }
      ty = d.node_type[n];
      if (ty == 1) {  // the wall projection is symmetric
        const double nx = d.node_n[2 * n], ny = d.node_n[2 * n + 1], dn = Db[0] * nx + Db[1] * ny;
        Db[0] -= dn * nx;
        Db[1] -= dn * ny;
      }
      p0 = d.v2e_ptr[n];
      p1 = d.v2e_ptr[n + 1];
      tk0 = d.nt[n];
      tk1 = d.ntn[n];
    }
    // displacement of each Voronoi element's vertex over [tau0, tau1]
    auto disp = [&](int j, int k, double* D) {
      D[0] = D[1] = 0.0;
      const long long dtj = d.dt[j];
      if (dtj <= 0) return;
      const double idtj = 1.0 / (double)dtj;
      const double tau0 = (double)(tk0 - d.t[j]) * idtj, tau1 = (double)(tk1 - d.t[j]) * idtj;
      const double* vd = d.vdisp + ((size_t)j * 3 + k) * 2 * Nt;
      const double dts = (double)dtj * d.etick[j];
      for (int c = 0; c < 2; ++c) {
        double a0 = vd[c * Nt + Nt - 1], a1 = a0;
        for (int pp = Nt - 2; pp >= 0; --pp) {
          a0 = a0 * tau0 + vd[c * Nt + pp];
          a1 = a1 * tau1 + vd[c * Nt + pp];
        }
        D[c] = dts * (a1 * tau1 - a0 * tau0);
      }
    };
    // a zero position adjoint contributes exact zeros
    const bool work = live && ty != 2 && (Db[0] != 0.0 || Db[1] != 0.0);
    double num0 = 0.0, num1 = 0.0, den = 0.0;
    if (work)
      for (int p = p0 + lane; p < p1; p += GS) {
        const int j = d.v2e[p];
        const double mu = d.Q[4 * (size_t)j] * adj::tri_area(d.X + 6 * (size_t)j);
        double D[2];
        disp(j, d.v2e_loc[p], D);
        num0 += mu * D[0];
        num1 += mu * D[1];
        den += mu;
      }
#pragma unroll
    for (int off = GS / 2; off > 0; off >>= 1) {
      num0 += __shfl_xor_sync(0xffffffffu, num0, off, GS);
      num1 += __shfl_xor_sync(0xffffffffu, num1, off, GS);
      den += __shfl_xor_sync(0xffffffffu, den, off, GS);
    }
    if (!work) continue;
    const double iden = 1.0 / den, D0 = num0 * iden, D1 = num1 * iden;
    const double n0b = Db[0] * iden, n1b = Db[1] * iden, denb = -(Db[0] * D0 + Db[1] * D1) * iden;
    for (int p = p0 + lane; p < p1; p += GS) {
      const int j = d.v2e[p], k = d.v2e_loc[p];
      const double* X = d.X + 6 * (size_t)j;
      const double rho = d.Q[4 * (size_t)j], area = adj::tri_area(X), mu = rho * area;
      double D[2];
      disp(j, k, D);
      const double mub = n0b * D[0] + n1b * D[1] + denb;
      atomicAdd(&a.Qb[4 * (size_t)j], mub * area);
      double Xb[6] = {0, 0, 0, 0, 0, 0};
      adj::tri_area_rev(X, mub * rho, Xb);
      for (int c = 0; c < 6; ++c) atomicAdd(&a.Xb[6 * (size_t)j + c], Xb[c]);
      const long long dtj = d.dt[j];
      if (dtj > 0) {
        // D = dts (sum_p vd[p] tau1^(p+1) - sum_p vd[p] tau0^(p+1)); element j's
        // vertex k is this node only, so its slot has one writer
        const double idtj = 1.0 / (double)dtj;
        const double tau0 = (double)(tk0 - d.t[j]) * idtj, tau1 = (double)(tk1 - d.t[j]) * idtj;
        const double dts = (double)dtj * d.etick[j];
        double* vdb = a.vdb + ((size_t)j * 3 + k) * 2 * Nt;
        double pw1 = tau1, pw0 = tau0;
        for (int pp = 0; pp < Nt; ++pp) {
          vdb[pp] += n0b * mu * dts * (pw1 - pw0);
          vdb[Nt + pp] += n1b * mu * dts * (pw1 - pw0);
          pw1 *= tau1;
          pw0 *= tau0;
        }
      }
    }
  }
}

// one launch copying several 8-byte arrays (the state arrays of a snapshot)
struct CopyList {
  const unsigned long long* src[16];
  unsigned long long* dst[16];
  long long n[16];
  int count;
};

// 16-byte words where both arrays allow them, four loads in flight per
// thread before their stores; the odd tail word (and unaligned arrays) by
// 8-byte words
__global__ void k_multi_copy(CopyList cl) {
  const long long nthr = (long long)gridDim.x * blockDim.x;
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  constexpr int U = 4;
  for (int k = 0; k < cl.count; ++k) {
    const unsigned long long* __restrict__ s = cl.src[k];
    unsigned long long* __restrict__ dd = cl.dst[k];
    const long long n = cl.n[k];
    long long done = 0;
    if ((((uintptr_t)s | (uintptr_t)dd) & 15) == 0) {
      const long long n2 = n / 2;
      const ulonglong2* __restrict__ s2 = reinterpret_cast<const ulonglong2*>(s);
      ulonglong2* __restrict__ d2 = reinterpret_cast<ulonglong2*>(dd);
      long long i = tid;
      for (; i + (U - 1) * nthr < n2; i += U * nthr) {
        ulonglong2 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) v[u] = s2[i + u * nthr];
#pragma unroll
        for (int u = 0; u < U; ++u) d2[i + u * nthr] = v[u];
      }
      for (; i < n2; i += nthr) d2[i] = s2[i];
      done = 2 * n2;
    }
    for (long long i = done + tid; i < n; i += nthr) dd[i] = s[i];
  }
}

__global__ void k_adj_reset(Counters* c, const Counters* saved) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int epoch = c->epoch;
  const int err = c->err_code, erre = c->err_elem;
  if (saved) *c = *saved;
  c->epoch = epoch + 1;  // epochs only grow: no stale stamp can match
  c->err_code = err;
  c->err_elem = erre;
  c->n_ready = 0;
  c->n_moved = 0;
  c->n_active = 0;
  c->n_touched = 0;
  c->n_cand[0] = c->n_cand[1] = 0;
  c->cand_valid = 0;
  c->finish_blocks = 0;
}

// d J / d(initial node positions): the node array's adjoint plus every
// element corner's adjoint (corner = node + a fixed periodic offset)
__global__ void k_adj_grad(Dev d, Adj a, double* gxy) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < d.ne; i += gridDim.x * blockDim.x)
    for (int k = 0; k < 3; ++k) {
      const int n = d.tri[3 * (size_t)i + k];
      atomicAdd(&gxy[2 * n], a.Xb[6 * (size_t)i + 2 * k]);
      atomicAdd(&gxy[2 * n + 1], a.Xb[6 * (size_t)i + 2 * k + 1]);
    }
}

template <int M>
void elem_impl(const Tab& T, const Dev& post, const Dev& live, const Adj& a, int nsm, cudaStream_t s, int initial) {
  constexpr size_t bytes = sizeof(ElemWork<M>);
  static_assert(bytes <= 227 * 1024, "element work space exceeds shared memory");
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_adj_elem<M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    cudaFuncSetAttribute(k_adj_elem<M>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
    attr = true;
  }
  const int per_sm = std::min(4, (int)((227 * 1024) / (bytes + 1024)));
  const int grid = initial ? post.ne : nsm * (per_sm > 0 ? per_sm : 1);
  k_adj_elem<M><<<grid, kElemThreads, bytes, s>>>(T, post, live, a, initial);
}

template <int M>
void phase_a_impl(const Tab& T, const Dev& live, const Dev& post, const Adj& a, int nsm, cudaStream_t s) {
  k_adj_commit<<<nsm * 2, 128, 0, s>>>(live, a);
  k_adj_update<<<nsm * 2, 128, 0, s>>>(live, post, a);
  k_adj_edges<M><<<nsm * 8, 128, 0, s>>>(T, live, a);
  k_adj_nodes_grp<<<nsm * 8, 128, 0, s>>>(T, live, a);
}

// ---------------------------------------------------------------------------
// host self-test of the element-level reverses (central differences)
// ---------------------------------------------------------------------------
struct Rng {
  unsigned long long s;
  double uni() {  // splitmix64 -> [0, 1)
    unsigned long long z = (s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    z ^= z >> 31;
    return (double)(z >> 11) * (1.0 / 9007199254740992.0);
  }
  double sym() { return 2.0 * uni() - 1.0; }
};

// fourth-order central difference of J at 0
template <class F>
double fd4(F& J, double e) {
  return (8.0 * (J(e) - J(-e)) - (J(2 * e) - J(-2 * e))) / (12.0 * e);
}

// smooth, physical test field (density, velocity, pressure) at (x, y)
void field(double x, double y, double* q) {
  const double rho = 1.0 + 0.2 * sin(1.3 * x + 0.4) * cos(0.9 * y - 0.2);
  const double u = 0.3 * cos(0.7 * x + 1.1 * y), v = -0.2 * sin(0.8 * x - 0.5 * y);
  const double p = 1.0 + 0.15 * cos(1.1 * x) * sin(0.6 * y + 0.3);
  q[0] = rho;
  q[1] = rho * u;
  q[2] = rho * v;
  q[3] = p / 0.4 + 0.5 * rho * (u * u + v * v);
}

template <int M>
double selftest_recon(const Tab& T, Rng& g) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc, NE = S::NE, NU = S::NU;
  auto* in = new adj::ReconIn<M>();
  auto* tp = new adj::ReconTape<M>();
  const double h = 0.1;
  // element: a perturbed equilateral triangle of size h around the origin
  const double base[6] = {0.0, 0.0, h, 0.0, 0.5 * h, 0.866 * h};
  for (int k = 0; k < 6; ++k) in->X[k] = base[k] + 0.1 * h * g.sym();
  const double cx = (in->X[0] + in->X[2] + in->X[4]) / 3, cy = (in->X[1] + in->X[3] + in->X[5]) / 3;
  field(cx, cy, in->Q);
  in->nU = 3 * NE;
  for (int u = 0; u < in->nU; ++u) {
    const double ang = 6.2831853 * g.uni(), r = h * (0.8 + 2.0 * g.uni());
    const double mx = cx + r * cos(ang), my = cy + r * sin(ang);
    for (int k = 0; k < 3; ++k) {
      in->Xv[u][2 * k] = mx + base[2 * k] - 0.5 * h + 0.1 * h * g.sym();
      in->Xv[u][2 * k + 1] = my + base[2 * k + 1] - 0.3 * h + 0.1 * h * g.sym();
    }
    field(mx, my, in->Qv[u]);
  }
  for (int s = 0; s < kNSten; ++s) {
    in->ok[s] = 1;
    in->st[s][0] = 0;
    for (int m = 1; m < NE; ++m) in->st[s][m] = (unsigned char)(1 + (s * 3 + m * 5) % in->nU);
  }
  double wb[Mc][4];
  for (int s = 0; s < Mc; ++s)
    for (int v = 0; v < 4; ++v) wb[s][v] = g.sym();
  // direction
  double dX[6], dQ[4];
  auto* dXv = new double[in->nU][6];
  auto* dQv = new double[in->nU][4];
  for (int k = 0; k < 6; ++k) dX[k] = h * g.sym();
  for (int v = 0; v < 4; ++v) dQ[v] = g.sym();
  for (int u = 0; u < in->nU; ++u) {
    for (int k = 0; k < 6; ++k) dXv[u][k] = h * g.sym();
    for (int v = 0; v < 4; ++v) dQv[u][v] = g.sym();
  }
  const adj::TeamSerial tm;
  adj::recon_fwd<M>(T, *in, *tp, tm);
  double Xb[6] = {0}, Qb[4] = {0};
  auto* Xvb = new double[in->nU][6]();
  auto* Qvb = new double[in->nU][4]();
  auto* rr = new adj::ReconRev<M>();
  adj::recon_rev<M>(T, *in, *tp, wb, Xb, Qb, Xvb, Qvb, *rr, tm);
  delete rr;
  double ad = 0.0;
  for (int k = 0; k < 6; ++k) ad += Xb[k] * dX[k];
  for (int v = 0; v < 4; ++v) ad += Qb[v] * dQ[v];
  for (int u = 0; u < in->nU; ++u) {
    for (int k = 0; k < 6; ++k) ad += Xvb[u][k] * dXv[u][k];
    for (int v = 0; v < 4; ++v) ad += Qvb[u][v] * dQv[u][v];
  }
  auto J = [&](double eps) {
    auto* p = new adj::ReconIn<M>(*in);
    for (int k = 0; k < 6; ++k) p->X[k] += eps * dX[k];
    for (int v = 0; v < 4; ++v) p->Q[v] += eps * dQ[v];
    for (int u = 0; u < p->nU; ++u) {
      for (int k = 0; k < 6; ++k) p->Xv[u][k] += eps * dXv[u][k];
      for (int v = 0; v < 4; ++v) p->Qv[u][v] += eps * dQv[u][v];
    }
    auto* t2 = new adj::ReconTape<M>();
    adj::recon_fwd<M>(T, *p, *t2, tm);
    double acc = 0.0;
    for (int s = 0; s < Mc; ++s)
      for (int v = 0; v < 4; ++v) acc += wb[s][v] * t2->w[s][v];
    delete t2;
    delete p;
    return acc;
  };
  const double e = 1e-5;
  const double fd = fd4(J, e);
  delete[] dXv; delete[] dQv; delete[] Xvb; delete[] Qvb;
  delete in; delete tp;
  (void)NU;
  return fabs(fd - ad) / fmax(fabs(fd), 1e-300);
}

template <int M>
double selftest_pred(const Tab& T, Rng& g) {
  using S = Sz<M>;
  constexpr int Mc = S::Mc;
  const double h = 0.1, dts = 0.02;
  double X[6] = {0.0, 0.0, h, 0.0, 0.5 * h, 0.866 * h}, w[Mc][4];
  for (int k = 0; k < 6; ++k) X[k] += 0.1 * h * g.sym();
  for (int s = 0; s < Mc; ++s) {
    const double x = X[0] + (X[2] - X[0]) * T.lat[s][0] + (X[4] - X[0]) * T.lat[s][1];
    const double y = X[1] + (X[3] - X[1]) * T.lat[s][0] + (X[5] - X[1]) * T.lat[s][1];
    field(5.0 * x, 5.0 * y, w[s]);
  }
  auto* tb = new adj::PredTables<M>();
  for (size_t k = 0; k < sizeof(adj::PredTables<M>) / sizeof(double); ++k) (&tb->tr[0][0][0][0])[k] = g.sym();
  double dX[6], dw[Mc][4];
  for (int k = 0; k < 6; ++k) dX[k] = h * g.sym();
  for (int s = 0; s < Mc; ++s)
    for (int v = 0; v < 4; ++v) dw[s][v] = g.sym();
  const adj::TeamSerial tm;
  auto* tp = new adj::PredTape<M>();
  auto* out = new adj::PredTables<M>();
  auto* pw = new adj::PredWork<M>();
  auto* pr = new adj::PredRev<M>();
  adj::pred_fwd<M>(T, T.nit, w, X, dts, *tp, *out, *pw, tm);
  double wb[Mc][4] = {}, Xb[6] = {0};
  adj::pred_rev<M>(T, T.nit, dts, *tp, *tb, wb, Xb, *pr, tm);
  double ad = 0.0;
  for (int k = 0; k < 6; ++k) ad += Xb[k] * dX[k];
  for (int s = 0; s < Mc; ++s)
    for (int v = 0; v < 4; ++v) ad += wb[s][v] * dw[s][v];
  auto J = [&](double eps) {
    double X2[6], w2[Mc][4];
    for (int k = 0; k < 6; ++k) X2[k] = X[k] + eps * dX[k];
    for (int s = 0; s < Mc; ++s)
      for (int v = 0; v < 4; ++v) w2[s][v] = w[s][v] + eps * dw[s][v];
    auto* t2 = new adj::PredTape<M>();
    auto* o2 = new adj::PredTables<M>();
    adj::pred_fwd<M>(T, T.nit, w2, X2, dts, *t2, *o2, *pw, tm);
    double acc = 0.0;
    for (size_t k = 0; k < sizeof(adj::PredTables<M>) / sizeof(double); ++k)
      acc += (&tb->tr[0][0][0][0])[k] * (&o2->tr[0][0][0][0])[k];
    delete t2;
    delete o2;
    return acc;
  };
  const double e = 1e-5;
  const double fd = fd4(J, e);
  delete tb; delete tp; delete out; delete pw; delete pr;
  return fabs(fd - ad) / fmax(fabs(fd), 1e-300);
}

template <int M>
double selftest_edge(const Tab& T, Rng& g, int has_R, int bc) {
  constexpr int Nt = M + 1;
  adj::EdgeIn<M> in;
  const double P0[4][2] = {{0.0, 0.0}, {0.1, 0.01}, {0.105, 0.014}, {0.004, 0.003}};
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 2; ++c) in.P[k][c] = P0[k][c] + 0.002 * g.sym();
  in.tk[0] = 100; in.tk[1] = 120; in.tk[2] = 180; in.tk[3] = 160;
  in.tsec = 1e-4;
  in.tL = 90; in.dtL = 100; in.tR = 110; in.dtR = 80;
  in.has_R = has_R;
  in.bc = bc;
  field(0.2, 0.15, in.qg);
  in.qg[3] *= 1.6;  // a hotter outer state: no tie of the two wave speeds
  for (int gx = 0; gx < Nt; ++gx) {
    double qa[4], qb[4];
    field(0.3 * gx, 0.1, qa);
    field(0.3 * gx + 0.05, 0.12, qb);
    for (int v = 0; v < 4; ++v) {
      in.trL[gx][0][v] = qa[v];
      in.trR[gx][0][v] = qb[v];
      for (int p = 1; p < Nt; ++p) {
        in.trL[gx][p][v] = 0.05 * g.sym() * qa[v];
        in.trR[gx][p][v] = 0.05 * g.sym() * qb[v];
      }
    }
  }
  double Gb[4], dP[4][2], dL[Nt][Nt][4], dR[Nt][Nt][4], dg[4];
  for (int v = 0; v < 4; ++v) Gb[v] = g.sym();
  for (int v = 0; v < 4; ++v) dg[v] = 0.1 * g.sym() * in.qg[v];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 2; ++c) dP[k][c] = 0.01 * g.sym();
  for (int k = 0; k < Nt * Nt * 4; ++k) {
    (&dL[0][0][0])[k] = g.sym();
    (&dR[0][0][0])[k] = g.sym();
  }
  double Pb[4][2] = {}, trLb[Nt][Nt][4] = {}, trRb[Nt][Nt][4] = {}, qgb[4] = {};
  adj::edge_rev<M>(T, in, Gb, Pb, trLb, trRb, qgb);
  double ad = 0.0;
  for (int v = 0; v < 4; ++v) ad += qgb[v] * dg[v];
  for (int k = 0; k < 4; ++k)
    for (int c = 0; c < 2; ++c) ad += Pb[k][c] * dP[k][c];
  for (int k = 0; k < Nt * Nt * 4; ++k) ad += (&trLb[0][0][0])[k] * (&dL[0][0][0])[k] + (&trRb[0][0][0])[k] * (&dR[0][0][0])[k];
  auto J = [&](double eps) {
    adj::EdgeIn<M> p = in;
    for (int k = 0; k < 4; ++k)
      for (int c = 0; c < 2; ++c) p.P[k][c] += eps * dP[k][c];
    for (int v = 0; v < 4; ++v) p.qg[v] += eps * dg[v];
    for (int k = 0; k < Nt * Nt * 4; ++k) {
      (&p.trL[0][0][0])[k] += eps * (&dL[0][0][0])[k];
      (&p.trR[0][0][0])[k] += eps * (&dR[0][0][0])[k];
    }
    double G[4];
    adj::edge_fwd<M>(T, p, G);
    return Gb[0] * G[0] + Gb[1] * G[1] + Gb[2] * G[2] + Gb[3] * G[3];
  };
  const double e = 1e-5;
  const double fd = fd4(J, e);
  return fabs(fd - ad) / fmax(fabs(fd), 1e-300);
}

template <int M>
double selftest_node(Rng& g, int type) {
  constexpr int Nt = M + 1, nv = 6;
  adj::NodeElem<M> el[nv];
  for (int k = 0; k < nv; ++k) {
    el[k].rho = 1.0 + 0.3 * g.uni();
    const double a0 = 6.2831853 * k / nv, a1 = 6.2831853 * (k + 1) / nv;
    const double X[6] = {0.0, 0.0, 0.1 * cos(a0), 0.1 * sin(a0), 0.1 * cos(a1), 0.1 * sin(a1)};
    for (int c = 0; c < 6; ++c) el[k].X[c] = X[c] + 0.005 * g.sym();
    for (int c = 0; c < 2; ++c)
      for (int p = 0; p < Nt; ++p) el[k].vd[c][p] = g.sym() / (p + 1);
    el[k].tau0 = 0.2 * g.uni();
    el[k].tau1 = el[k].tau0 + 0.5 + 0.3 * g.uni();
    el[k].dts = k == 3 ? 0.0 : 0.01 * (1 + g.uni());
  }
  const double nrm[2] = {0.6, 0.8};
  double Db[2] = {g.sym(), g.sym()};
  double drho[nv], dX[nv][6], dvd[nv][2][Nt];
  for (int k = 0; k < nv; ++k) {
    drho[k] = g.sym();
    for (int c = 0; c < 6; ++c) dX[k][c] = 0.01 * g.sym();
    for (int c = 0; c < 2; ++c)
      for (int p = 0; p < Nt; ++p) dvd[k][c][p] = g.sym();
  }
  double rhob[nv] = {}, Xb[nv][6] = {}, vdb[nv][2][Nt] = {};
  adj::node_rev<M>(nv, el, type, nrm, Db, rhob, Xb, vdb);
  double ad = 0.0;
  for (int k = 0; k < nv; ++k) {
    ad += rhob[k] * drho[k];
    for (int c = 0; c < 6; ++c) ad += Xb[k][c] * dX[k][c];
    for (int c = 0; c < 2; ++c)
      for (int p = 0; p < Nt; ++p) ad += vdb[k][c][p] * dvd[k][c][p];
  }
  auto J = [&](double eps) {
    adj::NodeElem<M> p[nv];
    for (int k = 0; k < nv; ++k) {
      p[k] = el[k];
      p[k].rho += eps * drho[k];
      for (int c = 0; c < 6; ++c) p[k].X[c] += eps * dX[k][c];
      for (int c = 0; c < 2; ++c)
        for (int q = 0; q < Nt; ++q) p[k].vd[c][q] += eps * dvd[k][c][q];
    }
    double D[2];
    adj::node_fwd<M>(nv, p, type, nrm, D);
    return Db[0] * D[0] + Db[1] * D[1];
  };
  const double e = 1e-5;
  const double fd = fd4(J, e);
  return fabs(fd - ad) / fmax(fabs(fd), 1e-300);
}

template <int M>
void selftest_impl(const Tab& T, unsigned long long seed, double* report) {
  Rng g{seed};
  double r = 0, p = 0, e = 0, n = 0;
  for (int rep = 0; rep < 4; ++rep) {
    r = fmax(r, selftest_recon<M>(T, g));
    p = fmax(p, selftest_pred<M>(T, g));
    e = fmax(e, selftest_edge<M>(T, g, 1, -1));
    e = fmax(e, selftest_edge<M>(T, g, 0, 0));
    e = fmax(e, selftest_edge<M>(T, g, 0, 1));
    n = fmax(n, selftest_node<M>(g, 0));
    n = fmax(n, selftest_node<M>(g, 1));
  }
  report[0] = r;
  report[1] = p;
  report[2] = e;
  report[3] = n;
}

}  // namespace

void launch_adj_elem(const Tab& T, const Dev& post, const Dev& live, const Adj& a, int nsm, cudaStream_t s, int initial) {
  switch (T.M) {
    case 1: elem_impl<1>(T, post, live, a, nsm, s, initial); break;
    case 2: elem_impl<2>(T, post, live, a, nsm, s, initial); break;
    default: elem_impl<3>(T, post, live, a, nsm, s, initial); break;
  }
}

void launch_adj_phase_a(const Tab& T, const Dev& live, const Dev& post, const Adj& a, int nsm, cudaStream_t s) {
  switch (T.M) {
    case 1: phase_a_impl<1>(T, live, post, a, nsm, s); break;
    case 2: phase_a_impl<2>(T, live, post, a, nsm, s); break;
    default: phase_a_impl<3>(T, live, post, a, nsm, s); break;
  }
}

void launch_adj_reset(const Dev& d, const Counters* saved, cudaStream_t s) {
  k_adj_reset<<<1, 32, 0, s>>>(d.cnt, saved);
}

void launch_multi_copy(const void* const* src, void* const* dst, const long long* n8, int count, int nsm,
                       cudaStream_t s) {
  CopyList cl{};
  cl.count = count;
  for (int k = 0; k < count; ++k) {
    cl.src[k] = (const unsigned long long*)src[k];
    cl.dst[k] = (unsigned long long*)dst[k];
    cl.n[k] = n8[k];
  }
  k_multi_copy<<<nsm * 4, 256, 0, s>>>(cl);
}

void launch_adj_grad(const Dev& d, const Adj& a, double* gxy, int nsm, cudaStream_t s) {
  k_adj_grad<<<nsm * 4, 128, 0, s>>>(d, a, gxy);
}

int adjoint_selftest(const Tab& T, unsigned long long seed, double* report) {
  switch (T.M) {
    case 1: selftest_impl<1>(T, seed, report); break;
    case 2: selftest_impl<2>(T, seed, report); break;
    default: selftest_impl<3>(T, seed, report); break;
  }
  return 0;
}

}  // namespace aw
