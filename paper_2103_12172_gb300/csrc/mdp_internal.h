// Internal structures shared by the host plan and the CUDA kernels.
#pragma once
#include <cstdint>
#include <vector>
#include <string>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>
#include "mdp.h"

// The bounds-checked build (libmdp_checked.so) is compiled with MDP_CHECKED=1: every batched
// kernel validates its block's work item and the gamma indices it writes through (first violation
// in the status word as MDP_ERR_BOUNDS, the access skipped), and MDP_FAULT_INJECT is honoured.
#ifndef MDP_CHECKED
#define MDP_CHECKED 0
#endif

namespace mdp {

// Per-subdomain geometry, coefficients and table offsets (POD; copied to the device).
//
// Grid: nodes (m, n), x_m = ax0 + m h, y_n = ay0 + n h. M+ is the node rectangle
// [mlo, mhi] x [nlo, nhi]. gamma is the 2-node ring [mlo-1, mhi+1] x [nlo-1, nhi+1]
// minus [mlo+1, mhi-1] x [nlo+1, nhi-1]; the support of r = L w|M+ ("ring") is
// [mlo, mhi] x [nlo, nhi] minus [mlo+2, mhi-2] x [nlo+2, nhi-2].
// Sine modes q = 1..Nq along x (Nq = Nx - 1, Nx = nx - 1 cells). The tridiagonal
// unknowns along y are rows n = nfirst .. nfirst + Nt - 1 (matrix row i = n - nfirst).
struct SubDesc {
  int nx, ny, Nx, Nq;
  int mlo, mhi, nlo, nhi;
  int Px, Py;       // M+ nodes along x and y
  int G, R;         // |gamma| = 4(Px + Py), |ring| = 4 Px + 4 (Py - 4)
  int nfirst, Nt;   // first y row of the tridiagonal unknowns, and their count
  int i0;           // first stored matrix row of the partial sweeps: (nlo - 1) - nfirst
  int NYf;          // stored rows of the forward (projection) sweep: Nt - i0
  int n_modes, n_cols;
  int cplx;         // 1: complex factors (Sommerfeld AP), 0: real (Dirichlet AP)
  int ap_bc;
  int xsym;         // 1: mlo + mhi == Nx (subdomain centred along x): paired ring layout
  int Ph;           // xsym: pair units per dense ring row, Nx/2 - mlo + 1
  int R2;           // ring residual slots: R, or 8 Ph + 4 (Py - 4) with xsym
  int nrec;         // receiver row (nlo+1 .. nhi-1) or -1; receivers m = mlo+1 .. mhi-1
  int rows_fft;     // inverse transform of the gamma rows by FFT (Nx a power of 2, 2Nx <= 4096)
  int fpb;          // FFTs (columns) per block of the dense-row kernels: max(1, 1024 / (2 Nx))
  int leader;       // index of the subdomain owning this one's tables (itself unless deduplicated)
  int tc_cols;      // 1: the gamma columns of the middle rows are summed on the tensor cores (k_inv_cols_tc)
  double h, k;
  double x0, x1, y0, y1, ax0, ay0;
  double c0, c1, c2;  // 9-point coefficients: centre, edge, corner (Eq. FD_scheme)
  double dc0, dc1;    // their k-derivatives (the corner one is 0)
  long long fact_off;   // doubles: factor rows [Nq][Nt][FW], FW = 8 (complex) or 4 (real)
  long long piv_off;    // bytes: pivot flags [Nq][Nt]
  long long dT_off;     // doubles: dT_q/dk rows [Nq][Nt][6] (sub, diag, super; complex)
  long long sin_off;    // doubles: sin(pi j / Nx), j = 0 .. 2Nx-1, then (2/Nx) sin(pi j/Nx)
  long long geo_off;    // doubles: gamma geometry [G][4] = (owner, s, rho, side length)
  long long seg_off;    // doubles: per mode [Nq][5] = (rlo, rhi, frlo, frhi, itop): real rows of the
                        // factor table, real rows of the forward-sweep table, last swept row
  long long fs_off;     // doubles: projection forward-sweep table [Nq][NYf][FSW] (rows i0..)
  long long tcb_off;    // doubles: tensor-core sums: per 16 modes a 1 KiB block of the fp16 sine digits at the
                        // gamma columns, then as many at the adjoint's ring columns (one column further in)
                        // of the sines, in the shared-memory operand layout of k_inv_cols_tc
  long long out_off;    // complex elements: start of the subdomain's output block
  long long rec_off;    // complex elements: start of the receiver block [n_cols][Px - 2]
  int *dstatus;         // the plan's device status word (bounds-checked build: first error; else unused)
};

// One batch work item: columns [col0, col0 + ncols) of subdomain `sub`, with its
// workspace slices (offsets in doubles from the workspace base).
struct Item {
  int sub, col0, ncols, flags;   // flags: bit0 basis densities, bit1 real data path
  long long xi_off;   // basis densities [G][ncols] (real) / dxi/dk follows for the gradient
  long long r_off;    // ring residual [R][ncols] (real or complex)
  long long gr_off;   // forward sine transform of the 4 dense ring rows [4][Nq][ncols]
  long long y_off;    // mode-space field [Nq][NY][ncols]
  long long a_off;    // adjoint mode-space field [Nq][Nt][ncols] (gradient pass)
  long long s_off;    // gradient source on the ring [R][ncols] (complex)
  long long red_off;  // per-block partial sums of the k-gradient (gradient pass); in the projection,
                      // per column the largest biased exponent of the stored mode-space rows (int)
  long long io_off;   // complex elements: column col0 of this item in xi / out / cot / grad_xi
};

enum { ITEM_BASIS = 1, ITEM_REAL = 2 };

// Launch-time view of a list of items: a device array plus, for each kernel family,
// per-item prefix sums of blocks. A single item may be passed by value instead.
struct Batch {
  const Item *items;    // device array (nullptr: use `one`)
  const int *prefix;    // device array [n_items + 1] of block prefix sums for this kernel
  const int *order;     // device array [total_blocks]: the item-major block number that launch
                        // block b runs (nullptr: b itself); the sweeps run their longest first
  int n_items;
  int total_blocks;
  Item one;
  // ranges the bounds-checked build validates every block's item against: subdomains, workspace
  // doubles, table doubles, pivot-flag bytes, and complex elements of the output / density /
  // cotangent arrays of the call; the status word that records the first violation
  int n_subs;
  int grad;             // the items are laid out for the gradient pass
  long long ws_n, tab_n, piv_n, out_n;
  int *status;
};

constexpr int FSW = 24;  // doubles per forward-sweep table row
constexpr int TRI_WARPS = 1;  // warps (modes) per block of the per-mode sweep kernel k_tri
constexpr int FFT_POINTS = 4096;        // longest transform (2 Nx) of the dense-row FFT kernels (64 KiB)
constexpr int FFT_BLOCK_POINTS = 1024;  // complex values per block when 2 Nx is shorter: fpb = 1024 / (2 Nx)

// Host buffer of the plan's tables: page-locked (cudaMallocHost) for plans with a device, so
// that uploads (plan creation, mdp_plan_update_k) run at full link speed; plain heap memory for
// host-only plans, which make no CUDA call. Zero-filled on allocation.
template <class T>
struct HostBuf {
  T *p = nullptr;
  size_t n = 0;
  bool pinned = false;
  HostBuf() = default;
  HostBuf(const HostBuf &) = delete;
  HostBuf &operator=(const HostBuf &) = delete;
  ~HostBuf() { release(); }
  void release() {
    if (p) { if (pinned) cudaFreeHost(p); else std::free(p); }
    p = nullptr; n = 0; pinned = false;
  }
  bool alloc(size_t count, bool want_pinned) {
    release();
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    if (want_pinned && cudaMallocHost((void **)&p, bytes) == cudaSuccess) pinned = true;
    else { p = (T *)std::malloc(bytes); pinned = false; }
    if (!p) return false;
    std::memset((void *)p, 0, bytes);
    n = count;
    return true;
  }
  T *data() { return p; }
  const T *data() const { return p; }
  size_t size() const { return n; }
  T &operator[](size_t i) { return p[i]; }
  const T &operator[](size_t i) const { return p[i]; }
};

struct HostSub {
  SubDesc d;
  std::vector<int> gamma_nm;     // 2*G: (n, m) pairs, row-major order
  std::vector<int> owner;        // G
  std::vector<double> rho, s, L; // G
  // this subdomain's slices of the plan's host tables (written in place by the factorisation)
  double *fact = nullptr;        // [Nq][Nt][FW]
  uint8_t *piv = nullptr;        // [Nq][Nt]
  double *dT = nullptr;          // [Nq][Nt][6]
  double *fs = nullptr;          // [Nq][NYf][FSW]: projection forward-sweep table
  std::vector<int> seg;          // [Nq][5]: see SubDesc::seg_off
};

struct Wave {
  std::vector<Item> items;
  long long ws_doubles;
};

}  // namespace mdp

struct mdp_plan {
  unsigned flags = 0;
  int n_subs = 0;
  int device = -1;
  std::vector<mdp::HostSub> subs;
  mdp::HostBuf<double> host_tables;      // all factor / dT / sweep / sine / geometry tables
  mdp::HostBuf<uint8_t> host_piv;
  long long out_size = 0;
  long long rec_size = 0;
  int tile_cols = 256;                   // columns per work item
  int fft_block_points = mdp::FFT_BLOCK_POINTS;  // complex values per block of the dense-row FFT kernels
  int tri_stages = 2;                    // table rows the projection sweep stages ahead (2 or 4)
  long long ws_budget = 0;               // bytes of workspace
  // batch schedules: [S_PROJ] mdp_project_batch over every subdomain, [S_GRAD] mdp_ap_adjoint
  // (larger workspace), [S_BASIS] basis columns of the distinct subdomains only (MDP_PLAN_DEDUPE
  // with duplicates; else empty)
  std::vector<mdp::Wave> sched[3];
  std::vector<int> leader;               // per subdomain: the subdomain whose tables and basis columns it shares
  // device side
  mdp::SubDesc *d_subs = nullptr;
  double *d_tables = nullptr;
  uint8_t *d_piv = nullptr;
  double *d_ws = nullptr;
  long long ws_doubles = 0;
  int *d_status = nullptr;
  int *d_fstatus = nullptr;               // status word of the device factorisation
  int fft_smem = 16;                     // dynamic shared memory of the FFT kernels: max fpb * 2 Nx * 16 B
  int n_sm = 0;                          // multiprocessors of the plan's device (persistent grids)
  mdp::HostBuf<mdp::SubDesc> sub_stage;  // pinned copy of the subdomain descriptors (async upload)
  mdp::HostBuf<int> h_fstatus;           // pinned read-back of d_fstatus
  bool host_stale = false;               // device tables refactored since the host tables were built
  // second table set of mdp_plan_update_k_async (allocated by its first call). d_subs, d_tables
  // and d_piv name physical set `set`; the alt_* pointers the other. ready_ev[s]: after the last
  // refactorisation into set s; used_ev[s]: after the last compute call that read it.
  mdp::SubDesc *alt_subs = nullptr;
  double *alt_tables = nullptr;
  uint8_t *alt_piv = nullptr;
  mdp::HostBuf<mdp::SubDesc> alt_stage;  // pinned descriptor stage of set 1 (sub_stage: set 0)
  int set = 0;
  cudaEvent_t ready_ev[2] = {nullptr, nullptr};
  cudaEvent_t used_ev[2] = {nullptr, nullptr};
  bool used_rec[2] = {false, false};
  // per schedule and wave: device items and prefix arrays (one prefix array per kernel family)
  std::vector<mdp::Item *> d_items[3];
  std::vector<int *> d_order[3];         // [wave] -> device int [k_tri + k_adj_tri blocks]: launch orders
  std::vector<int *> d_prefix[3];        // [wave] -> device int [NFAM][n_items + 1]
  std::vector<std::vector<int>> h_prefix[3];
  // CUDA graphs of mdp_project_batch, keyed by (xi, out, kind, stream, table set)
  struct GraphEntry {
    const void *xi; void *out; void *out_rec; int kind; cudaStream_t st; const double *tab; cudaGraphExec_t exec;
  };
  std::vector<GraphEntry> graphs;
  // per-kernel event timing (mdp_plan_profile)
  bool prof_on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev[16];
  int prof_used[16] = {0};
};

namespace mdp {

enum Sched { S_PROJ = 0, S_GRAD = 1, S_BASIS = 2 };

// the ranges a launch's Batch carries for the bounds-checked build (out_n: complex elements of the
// call's output, density and cotangent arrays)
inline void set_bounds(const mdp_plan *p, Batch &b, long long out_n, bool grad) {
  b.n_subs = p->n_subs;
  b.grad = grad ? 1 : 0;
  b.ws_n = p->ws_doubles;
  b.tab_n = (long long)p->host_tables.size();
  b.piv_n = (long long)p->host_piv.size();
  b.out_n = out_n;
  b.status = p->d_status;
}

// kernel families (each has its own block decomposition of an item); F_A* are the adjoint's
enum Fam { F_EXT = 0, F_RES, F_FROWS, F_TRI, F_IROWS, F_ICOLS, F_AFWD, F_ATRI, F_ARING, F_ARINGC, F_AGAM, F_IREC,
           F_ACOLS, F_TCOLS, F_ATCOLS, NFAM };

// Blocks of kernel family f for an item of ncols columns: 32 columns (x) times BY tasks (y).
// The same function numbers the blocks on the host (prefix sums) and in the kernels.
inline __host__ __device__ int blocks_for(int f, const SubDesc &d, int ncols) {
  const int cb = (ncols + 31) / 32;
  switch (f) {
    case F_EXT: return (d.G + 127) / 128;
    case F_RES: return cb * (((d.xsym ? 4 * d.Ph + 2 * (d.Py - 4) : d.R) + 7) / 8);
    case F_FROWS:
      if (d.rows_fft) return 4 * ((ncols + d.fpb - 1) / d.fpb);
      return cb * ((d.Nx / 2 + 7) / 8);
    case F_TRI: return cb * ((d.Nq + TRI_WARPS - 1) / TRI_WARPS);
    case F_IROWS:
      if (d.rows_fft) return 4 * ((ncols + d.fpb - 1) / d.fpb);
      return cb * (((d.xsym ? 4 * (d.Ph + 1) : 4 * (d.Px + 2)) + 7) / 8);
    case F_ICOLS: return d.tc_cols ? 0 : cb * ((d.Py - 2 + 7) / 8);
    case F_TCOLS: return d.tc_cols ? ((ncols + 63) / 64) * (d.Py - 2) : 0;   // tiles: middle row x 64 columns
    case F_AFWD:
      if (d.rows_fft) return 5 * ((ncols + d.fpb - 1) / d.fpb);
      return cb * ((d.Nx / 2 + 7) / 8);
    case F_ATRI: return cb * ((d.Nq + 3) / 4);
    case F_ARING:
      if (d.rows_fft) return 4 * ((ncols + d.fpb - 1) / d.fpb);
      return cb * ((4 * d.Px + 7) / 8);
    case F_ARINGC: return d.tc_cols ? 0 : cb * ((d.Py - 4 + 7) / 8);
    case F_ATCOLS: return d.tc_cols && d.Py > 4 ? ((ncols + 63) / 64) * (d.Py - 4) : 0;   // tiles: inner middle row x 64 columns
    case F_AGAM: return cb * ((d.G + 7) / 8);
    case F_IREC: return d.nrec < 0 ? 0 : cb * (((d.xsym ? d.Ph - 1 : d.Px - 2) + 7) / 8);
    case F_ACOLS: return cb * ((d.Py - 2 + 7) / 8);
    default: return 0;
  }
}

// slot bases of the per-block gradient partials of an item: [ATRI | ARING | ARINGC or 4 per ATCOLS
// tile | AGAM], total
inline __host__ __device__ void red_slots(const SubDesc &d, int ncols, int base[5]) {
  base[0] = 0;
  base[1] = base[0] + blocks_for(F_ATRI, d, ncols);
  base[2] = base[1] + blocks_for(F_ARING, d, ncols);
  base[3] = base[2] + blocks_for(F_ARINGC, d, ncols) + 4 * blocks_for(F_ATCOLS, d, ncols);
  base[4] = base[3] + blocks_for(F_AGAM, d, ncols);
}
// Workspace slices of an item of ncols columns, in doubles from the item's base (each 256-byte
// aligned): basis densities, ring residual, dense-row transforms, mode-space field, and for the
// gradient pass the adjoint field, k-source and per-block partials; the last slice holds per
// column the largest biased exponent (ints) of the kept mode-space rows (projection) or of the
// adjoint field's inner middle rows (gradient pass, after the partials and their total).
inline __host__ __device__ void item_workspace(const SubDesc &d, int ncols, bool grad, long long &xi, long long &r,
                                               long long &gr, long long &y, long long &a, long long &s,
                                               long long &red, long long &total) {
  auto al = [](long long v) { return (v + 31) & ~31LL; };
  long long off = 0;
  xi = off; off += al((long long)d.G * ncols * (grad ? 2 : 1));
  r = off;  off += al((long long)(d.R > d.R2 ? d.R : d.R2) * ncols * 2);
  gr = off; off += al(5LL * d.Nq * ncols * 2);  // 4 dense rows (+ the receiver row in the adjoint)
  y = off;  off += al((long long)d.Nq * (grad ? d.Nt : d.NYf) * ncols * 2);
  a = off;  off += grad ? al((long long)d.Nq * d.Nt * ncols * 2) : 0;
  s = off;  off += grad ? al((long long)d.R * ncols * 2) : 0;
  int rs[5];
  red_slots(d, ncols, rs);
  red = off; off += grad ? al(rs[4] + 1 + (ncols + 1) / 2) : al((ncols + 1) / 2);
  total = off;
}
const char *fam_name(int f);
// event pair around a launch when profiling is on
void prof_begin(mdp_plan *p, int fam, cudaStream_t st);
void prof_end(mdp_plan *p, int fam, cudaStream_t st);
// plan construction (host)
mdp_status build_host_plan(mdp_plan *p, const mdp_subdomain *subs, int n);
mdp_status refactor_host(mdp_plan *p, const double *k);
mdp_status set_k_fields(mdp_plan *p, const double *k);   // validate k, update the k-dependent SubDesc fields
cudaError_t launch_factor(const mdp_plan *p, int *status, cudaStream_t st);   // factor.cu
// the same into an explicit table set (descriptors ds, tables tab, pivot flags piv)
cudaError_t launch_factor_to(const mdp_plan *p, const SubDesc *ds, double *tab, uint8_t *piv, int *status,
                             cudaStream_t st);
void host_mode_solve(const HostSub &hs, int q, int adjoint, const double *b, double *x);
// kernel launchers (kernels.cu)
enum { PASS_FWD = 0, PASS_GRAD = 1 };
cudaError_t set_kernel_attributes();      // kernels.cu: opt-in shared memory of the FFT kernels
cudaError_t set_adj_kernel_attributes();  // kernels_adj.cu
cudaError_t set_tc_kernel_attributes();   // kernels_tc.cu
// the gamma columns of the middle rows on the tensor cores (items whose subdomain has tc_cols)
cudaError_t launch_inv_cols_tc(const Batch &b, const SubDesc *subs, const double *tab, const double *ws,
                               const double2 *xi_user, double2 *out, int kind, int *status, int n_sm,
                               cudaStream_t st);
// the adjoint's sums at the 4 ring columns of the inner middle rows (dk: with the k-gradient partials)
cudaError_t launch_adj_cols_tc(const Batch &b, const SubDesc *subs, const double *tab, double *ws, bool dk,
                               int *status, int n_sm, cudaStream_t st);
cudaError_t launch_project(mdp_plan *p, const Batch *fam_batches, int out_kind, const double2 *xi_user,
                           double2 *out, double2 *out_rec, cudaStream_t st);
cudaError_t launch_adjoint(mdp_plan *p, const Batch *fam_batches, int out_kind, const double2 *xi_user,
                           const double2 *cot, const double2 *cot_rec, double2 *grad_xi, double *grad_k,
                           cudaStream_t st);
// the adjoint's own kernels (kernels_adj.cu), after the forward recompute of the gradient pass
cudaError_t launch_adjoint_tail(mdp_plan *p, const Batch *fb, int out_kind, const double2 *xi_user, const double2 *cot,
                                const double2 *cot_rec, double2 *grad_xi, double *grad_k, cudaStream_t st);

cudaError_t launch_potential(const mdp_plan *p, int sub, int ncols, const double2 *xi, double2 *u, cudaStream_t st);
cudaError_t launch_source_terms(mdp_plan *p, int sub, const double2 *f, const double2 *src4, double2 *F, double2 *u,
                                cudaStream_t st);
cudaError_t launch_basis_densities(const mdp_plan *p, int sub, int col0, int ncols, double2 *out, cudaStream_t st);
cudaError_t launch_solve(const mdp_plan *p, int sub, int nrhs, const double2 *g, double2 *u, int adjoint,
                         cudaStream_t st);
cudaError_t launch_solve_raw(const SubDesc *d_sub, const SubDesc &hd, const double *tab, const uint8_t *piv,
                             double *buf, long long buf_doubles, int nrhs, const double2 *g, double2 *u, int adjoint,
                             cudaStream_t st);
}  // namespace mdp
