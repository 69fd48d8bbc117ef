// Internal declarations shared by the host driver and the kernels of the
// GB300 library (not part of the C ABI).
#pragma once
#include <cstdint>

#include <cuda_runtime.h>

namespace aw {

constexpr int kMaxM = 3;
constexpr int kMaxMc = 10;   // (M+1)(M+2)/2
constexpr int kMaxNt = 4;    // M+1 Gauss-Lobatto times
constexpr int kMaxNU = 9;    // Mc - 1 non-constant basis functions
constexpr int kMaxNe = 20;   // stencil size n_e = 2 Mc
constexpr int kNSten = 7;    // central + 3 primary + 3 reverse sectors

// Reference tables of one order M, built on the host at context creation and
// passed to kernels by value (uniform reads broadcast from the parameter bank).
struct Tab {
  int M, Mc, Nt, Nst, NU;
  double gamma, cfl, tick;
  long long T;          // t_end in ticks
  int eulerian;         // mesh velocity V = 0
  int gts;              // global time step
  int nit;              // Picard iterations
  int flux;             // 0 Rusanov-type, 1 Osher-type ALE flux
  double wall_u, wall_v, wall_speed;  // moving slip walls (boundary tag 2)
  long long Tsw;        // ticks of the global-step start-up (0: none)
  double cfl_start;     // its CFL number
  double kidder[5];     // r_i0, r_e0, rho_i0, rho_e0, s0 of the Kidder state (boundary tag 3)
  double lat[kMaxMc][2];
  int vnode[3];
  double Dxi[kMaxMc][kMaxMc], Deta[kMaxMc][kMaxMc];
  double B[kMaxNt - 1][kMaxNt];   // qhat_t = qhat_0 + dt * sum_t' B[t-1][t'] P_t'
  double Dtau[kMaxNt][kMaxNt];
  double VtInv[kMaxNt][kMaxNt];   // monomial coefficients in tau from slice values
  double Tr[3][kMaxNt][kMaxMc];   // Lagrange basis at the Gauss points of each local edge
  double wavg[kMaxMc];            // reference-triangle average of each Lagrange function
  double Bnod[kMaxMc][kMaxNU];    // zero-mean centred monomials at the lattice nodes
  int mexp[kMaxNU][2];
  double mbar[kMaxNU];
  double SigU[kMaxNU][kMaxNU];    // upper Cholesky factor: sigma = |SigU c|^2
  double glx[kMaxNt], glw[kMaxNt];
};

// Device-resident context data (pointers into one context's allocations).
struct Dev {
  int ne, nn, ned, periodic;
  double period[2];
  // mesh
  const int* tri;          // [ne*3]
  const double* cshift;    // [ne*6] corner image offsets (shift * period)
  const int* elem_edge;    // [ne*3]
  const int* edge_nodes;   // [ned*2]
  const int* edge_elem;    // [ned*2]
  const signed char* edge_loc;  // [ned*2]
  const signed char* edge_bc;   // [ned]
  const int* nbr;          // [ne*3]
  const double* nbr_shift; // [ne*6]
  const int* n2e_ptr;      // [nn+1] node -> incident edges
  const int* n2e;
  const int* v2e_ptr;      // [nn+1]
  const int* v2e;          // node -> element
  const signed char* v2e_loc;
  const signed char* node_type;
  const double* node_n;    // [nn*2]
  const int* sw_ptr;       // [ne+1]
  const int* sw;
  const int* u_ptr;        // [ne+1] unique stencil members (without i)
  const int* u_elem;
  const double* u_shift;   // [2 per entry]
  const unsigned char* sten;  // [ne][7][n_e] local member index (0 = i itself)
  const signed char* sten_ok; // [ne*7]
  const double* etick;     // [ne] seconds per tick of the element's instance
  // element state
  double* Q;     // [ne*4]
  double* QM;    // [ne*4]
  double* HM;    // [ne*4] (x, y, t, pad)
  long long* t;  // [ne]
  long long* dt; // [ne]
  double* X;     // [ne*6]
  long long* count;
  double* qhat;  // [ne*Nst*4]
  double* trace; // [ne*3*Nt*Nt*4]: per edge, Gauss point, tau monomial, variable
  double* avgc;  // [ne*Nt*4]: tau monomial coefficients of the reference average
  double* vdisp; // [ne*3*2*Nt]: coefficients of int_0^tau V_h(vertex) (powers 1..Nt)
  // nodes
  double* nX;    // [nn*2]
  long long* nt; // [nn]
  double* nXn;   // [nn*2] new positions in the running sweep
  long long* ntn;
  // sweep scratch
  int* elem_ready;   // [ne] epoch stamp when ready
  int* elem_touch;   // [ne] epoch stamp when adjacent to an active edge
  int* node_moved;   // [nn] epoch stamp
  int* edge_act;     // [ned] epoch stamp
  int* ready_list;   // [ne]
  int* moved_list;   // [nn]
  int* active_list;  // [ned]
  int* touch_list;   // [ne]
  int* cand_stamp;   // [ne] epoch stamp when listed as a candidate
  int* cand_list;    // [2][ne] ready candidates of the next sweep (double buffer)
  double* G;         // [ned*4]
  double* N;         // [ned*4]
  double* w0;        // [ne*Mc*4] nodal WENO values, by position in the ready list
  struct Counters* cnt;
  // frozen schedule: 0 free, 1 record, 2 replay the dt ticks of each
  // element's update count c at sched_log[i * sched_k + c]
  long long* sched_log;
  long long sched_k;
  int sched_mode;
};

// Adjoint arrays (same layouts as the state they belong to).
struct Adj {
  double* Qb;    // [ne*4]
  double* QMb;   // [ne*4]
  double* Xb;    // [ne*6]
  double* trb;   // [ne*3*Nt*Nt*4]
  double* avb;   // [ne*Nt*4]
  double* vdb;   // [ne*6*Nt]
  double* nXb;   // [nn*2]
  double* nXnb;  // [nn*2] new node positions of the running sweep
  double* gb;    // [ne*4] adjoint multiplying -sign * G of each own edge
};

struct Counters {
  int epoch;
  int n_ready;
  int n_moved;
  int n_active;
  int n_touched;
  int n_unfinished;  // elements with t < t_sync (maintained across sweeps)
  int n_cand[2];
  int cand_valid;    // 0: the next sweep checks every element
  int err_code;
  int err_elem;
  unsigned long long gcl_bits;   // max GCL residual (non-negative double bits)
  long long gts_min;
  long long updates;             // total element updates
  long long sweeps;
  long long productive;           // sweeps that updated at least one element
  int last_ready;                 // ready elements of the last completed sweep
  int finish_blocks;
  long long updates_since_sync;
  long long surfaces;            // space-time edge surfaces integrated (all sweeps)
  long long t_sync;              // sync time in ticks: steps are clipped at it and elements
                                 // stop there (T unless aw_advance_to set an earlier time)
};

// Tile shapes of a sweep's kernels (they change no arithmetic): recon_half
// halves the reconstruction's elements and threads per block, pred_wide runs the
// predictor on 256-thread blocks instead of 128, bpsm = blocks per SM of the
// persistent kernels that loop over the sweep's lists.
struct Tiles {
  int recon_half = 0;
  int pred_wide = 0;
  int bpsm = 8;
};

// kernel launchers (aw_kernels.cu)
constexpr int kNumKernels = 8;  // launches per sweep
const char* kernel_name(int k);
// side, fork, join (optional, plain launches only): the node solver on the
// side stream, beside the edge marking on s
void launch_sweep(const Tab& tab, const Dev& d, int nsm, cudaStream_t s, cudaEvent_t* ev, const Tiles& tl,
                  cudaStream_t side = nullptr, cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
void launch_initial(const Tab& tab, const Dev& d, int nsm, cudaStream_t s, const Tiles& tl);
void launch_products(const Tab& tab, const Dev& d, int nsm, cudaStream_t s);
// a new sync time Tn below the current one: every step crossing Tn is cut back
// to it and its predictor re-solved from the element's own tau = 0 dofs
void launch_sync_cut(const Tab& tab, const Dev& d, int nsm, cudaStream_t s, long long Tn, const Tiles& tl);
// a new sync time above the current one Told: the elements stopped at Told get
// their phase B (reconstruction, step, predictor)
void launch_sync_resume(const Tab& tab, const Dev& d, int nsm, cudaStream_t s, long long Told, const Tiles& tl);
double measure_fp64_peak();
// k_ready, k_nodes, k_edges of one sweep: ready/moved/active/touched lists
// and the new node positions, without changing the state
void launch_phase_a_lists(const Tab& tab, const Dev& d, int nsm, cudaStream_t s);

// adjoint kernels (aw_adjoint.cu)
void launch_adj_elem(const Tab& tab, const Dev& post, const Dev& live, const Adj& a, int nsm, cudaStream_t s,
                     int initial);
void launch_adj_phase_a(const Tab& tab, const Dev& live, const Dev& post, const Adj& a, int nsm, cudaStream_t s);
// per-sweep counters to zero, candidates invalid, epoch + 1; with saved (a
// device copy of the counters) != 0 the other fields are copied from it
void launch_adj_reset(const Dev& d, const Counters* saved, cudaStream_t s);
void launch_adj_grad(const Dev& d, const Adj& a, double* gxy, int nsm, cudaStream_t s);
// copies count arrays of n8[k] 8-byte words from src[k] to dst[k] in one launch (count <= 16)
void launch_multi_copy(const void* const* src, void* const* dst, const long long* n8, int count, int nsm,
                       cudaStream_t s);
// host-side check of every element-level reverse against central
// differences of its forward; report[0..3]: recon, predictor, edge, node
int adjoint_selftest(const Tab& tab, unsigned long long seed, double* report);

}  // namespace aw

struct aw_ctx;
namespace aw {
// Makes a context's device current for the life of an entry point and gives
// the caller's device back afterwards: a context's stream, kernels, memory
// and graphs belong to the device that was current at aw_create.
class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (dev >= 0 && cudaGetDevice(&prev_) == cudaSuccess && prev_ != dev && cudaSetDevice(dev) == cudaSuccess)
      switched_ = true;
  }
  ~DeviceGuard() {
    if (switched_) cudaSetDevice(prev_);
  }
  DeviceGuard(const DeviceGuard&) = delete;
  DeviceGuard& operator=(const DeviceGuard&) = delete;

 private:
  int prev_ = -1;
  bool switched_ = false;
};

struct CtxView {
  const Dev* d;
  long long T;          // the sync time in ticks (elements at or beyond it are not updated)
  cudaStream_t stream;
  int device;           // the device of the context
};
// false if the context has no valid state
bool ctx_view(aw_ctx* c, CtxView* v);
void ctx_error(aw_ctx* c, const char* msg);
}  // namespace aw
