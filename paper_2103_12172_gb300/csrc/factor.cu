// Per-mode factorisation on the GPU: the tables that mdp_plan_update_k rebuilds for new
// wavenumbers (CUDA, sm_103a, FP64).
//
// For every subdomain and sine mode q the AP's y-direction system T_q (Section 3.2.1; the
// separable form of the 4th-order compact scheme) is factored by the pivoted banded LU, and
// the tables of the sweeps are written straight into the plan's device tables:
//   - factor rows (l, 1/d, du/d, du2/d), the swap flags and dT_q/dk rows (gradient pass,
//     full-grid solves), with the run of exactly-real rows around the middle row;
//   - the condensed, pivot-scaled forward-sweep rows of the projection (rows above the ring
//     folded into the last pivot by their Schur complement), with its run of real rows.
// The host plan builds the same tables at plan creation (plan.cpp: mode_matrix, band_lu,
// factor_mode, build_fs_mode). Two kernels:
//   k_factor_chain  the pivot recurrences, the only sequential part: one thread per (mode,
//                   table) streams the rows with O(1) state and stores each raw LU row (l, d,
//                   1/d, du, du2, swap) in place in its table row. A chain is a long sequence of
//                   dependent FP64 operations, so it does nothing else, and its interior
//                   no-swap steps take a real-coefficient fast path.
//   k_factor_rows   everything row-local, one block per mode: u1 = du/d, u2 = du2/d, the
//                   sweep rows (which also need row i+1's pivot, read through shared memory in
//                   chunks so the rows can be rewritten in place), the dT/dk rows, and the runs
//                   of exactly-real rows (block reductions).
#include "kernels_common.cuh"
#include "mdp_probe.h"

namespace mdp {
namespace {

constexpr double kSingularTolD = 1e-13;   // pivot below this x max|T| -> singular
constexpr double kCondenseTolD = 1e-8;    // Schur complement below this x max|T|: keep all rows

__device__ __forceinline__ double cabs2(cplx a) { return fma(a.re, a.re, a.im * a.im); }
__device__ __forceinline__ cplx cscale(double s, cplx a) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ bool czero(cplx a) { return a.re == 0.0 && a.im == 0.0; }
// 1/x for x > 0: a single-precision seed y0 (relative error below 2^-21) refined by one cubic
// step of the Newton-Raphson iteration for 1/x (Goldschmidt form): with e = 1 - x y0,
// 1/x = y0 / (1 - e) = y0 (1 + e + e^2) + O(e^3 y0), i.e. full double precision. Six dependent
// operations instead of a full division on the factorisation's serial chains; x outside the
// float range takes the division.
__device__ __forceinline__ double rcp_pos(double x) {
  if (!(x > 0x1p-120 && x < 0x1p120)) return 1.0 / x;
  const double y0 = (double)__fdividef(1.0f, (float)x);
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}
// 1/b and a/b through one real reciprocal of |b|^2 (the magnitudes here are O(1/h^2))
__device__ __forceinline__ cplx crecip(cplx b) {
  const double r = rcp_pos(cabs2(b));
  return {b.re * r, -b.im * r};
}
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) { return cmul(a, crecip(b)); }
// an entry whose imaginary part is below 2^-60 of its modulus is real to working precision
__device__ __forceinline__ bool tiny_im(cplx v) { return v.im * v.im <= 0x1p-120 * cabs2(v); }

// Entries of T_q (rows 0..N-1): dl(i) = T[i+1][i], dg(i) = T[i][i], du(i) = T[i][i+1]; interior
// rows (a, dd, a); with Sommerfeld rows (cplx) row 0 is (c_p, c_m) and row N-1 has diagonal c_p
// and sub-diagonal c_m, c_p = alpha + beta/2, c_m = -alpha + beta/2 (all scaled by 1/h).
struct ModeRows {
  int N;
  bool cplx_ap;
  double a, dd;           // interior entries
  cplx cp, cm;            // Sommerfeld row entries
  double da, ddd;         // their k-derivatives
  cplx tp, tm;            // k-derivatives of cp, cm
  __device__ void entries(int i, cplx &dl, cplx &dg, cplx &du) const {
    dl = cmk(a, 0.0); dg = cmk(dd, 0.0); du = cmk(a, 0.0);
    if (cplx_ap && i == 0) { dg = cp; du = cm; }
    if (cplx_ap && i == N - 1) dg = cp;
    if (cplx_ap && i == N - 2) dl = cm;
  }
  __device__ double scale2() const {   // max |T_ij|^2
    double s = fmax(a * a, dd * dd);
    if (cplx_ap) s = fmax(s, fmax(cabs2(cp), cabs2(cm)));
    return s;
  }
};

__device__ ModeRows mode_rows(const SubDesc &d, int q) {
  ModeRows m;
  m.N = d.Nt;
  m.cplx_ap = d.cplx != 0;
  const double h = d.h, h2 = h * h, k = d.k, k2 = k * k;
  const double sq = sin(M_PI * q / (2.0 * d.Nx));
  const double lam = -4.0 * sq * sq;   // eigenvalue of the second difference along x
  m.a = 1.0 / h2 + lam / (6.0 * h2) + k2 / 12.0;
  m.dd = -2.0 * m.a + lam / h2 + k2 + k2 * lam / 12.0;
  m.da = k / 6.0;
  m.ddd = -2.0 * m.da + 2.0 * k + 2.0 * k * lam / 12.0;
  const bool paper = d.ap_bc == MDP_AP_DIRX_SOMMY_PAPER;                   // the rows as printed
  const double alpha = paper ? (1.0 - k2 * h2 / 24.0 - lam / 6.0) / h2 : (1.0 + k2 * h2 / 24.0 + lam / 24.0) / h2;
  const double beta = k * (1.0 + k2 * h2 / 8.0 + lam / (paper ? 2.0 : 8.0)) / h;           // imaginary part
  const double dalpha = paper ? -k / 12.0 : k / 12.0;
  const double dbeta = (1.0 + 3.0 * k2 * h2 / 8.0 + lam / (paper ? 2.0 : 8.0)) / h;        // imaginary part
  m.cp = cmk(alpha, 0.5 * beta);
  m.cm = cmk(-alpha, 0.5 * beta);
  m.tp = cmk(dalpha, 0.5 * dbeta);
  m.tm = cmk(-dalpha, 0.5 * dbeta);
  return m;
}

// One step of the banded LU with partial pivoting, streamed: on entry (g, u) are the current
// diagonal and super-diagonal of row i, (lsub, gn, un) the original T[i+1][i], T[i+1][i+1],
// T[i+1][i+2]. On exit (l, dinv, dup, du2, sw) are row i's multiplier, inverse pivot, first and
// second super-diagonal of U and swap flag (the pivot itself is returned in dfin), and (g, u)
// hold row i+1. last2: i == n-2 (no du2 fill-in). Returns false on a zero pivot.
__device__ __forceinline__ bool lu_step(cplx &g, cplx &u, cplx lsub, cplx gn, cplx un, bool last2, cplx &l,
                                        cplx &dfin, cplx &dinv, cplx &dup, cplx &du2, uint8_t &sw) {
  if (cabs2(g) >= cabs2(lsub)) {
    if (czero(g)) return false;
    const cplx lu = cmul(lsub, u);   // off the g -> g' chain
    dinv = crecip(g);
    const cplx f = cmul(lsub, dinv);
    l = f; dfin = g; dup = u; du2 = cmk(0.0, 0.0); sw = 0;
    g = csub(gn, cmul(lu, dinv));
    u = un;
  } else {
    dinv = crecip(lsub);
    const cplx f = cmul(g, dinv);
    l = f; dfin = lsub; dup = gn; sw = 1;
    const cplx gnew = csub(u, cmul(f, gn));
    du2 = last2 ? cmk(0.0, 0.0) : un;
    u = last2 ? un : cscale(-1.0, cmul(f, un));
    g = gnew;
  }
  return true;
}

__device__ __forceinline__ void set_error(int *status, int code) { atomicCAS(status, 0, code); }

// Subdomain of mode number t over the modes of the subdomains that own their tables (duplicates
// share their leader's); t becomes the mode index within it. n_subs if t is past the end.
__device__ __forceinline__ int mode_owner(const SubDesc *subs, int n_subs, int &t) {
  int si = 0;
  for (; si < n_subs; ++si) {
    if (subs[si].leader != si) continue;
    if (t < subs[si].Nq) break;
    t -= subs[si].Nq;
  }
  return si;
}

// The pivoted LU of rows 0..n-1 of T_q (diagonal of row `mod` reduced by sigma), calling
// out(i, l, d, dinv, du, du2, sw) for every row in order. Interior steps (real a, dd entries,
// super-diagonal of the pivot row still the original a) that keep the pivot take the fast path
// with real coefficients. Returns false (status set) on a singular pivot.
template <class Out>
__device__ bool lu_chain(const ModeRows &M, int n, int mod, cplx sigma, double tol2, int *status, Out out) {
  const int N = M.N;
  auto ent = [&](int i, cplx &dl, cplx &dg, cplx &du) {
    M.entries(i, dl, dg, du);
    if (i == mod) dg = csub(dg, sigma);
  };
  const double a = M.a, dd = M.dd, a2 = M.a * M.a;
  // steps i < fast_end have T[i+1][i] = a and T[i+1][i+1] = dd (not a Sommerfeld row, not the
  // reduced row); they take the fast path while the pivot row's super-diagonal is still a
  const int fast_end = min(M.cplx_ap ? N - 2 : n - 1, mod - 1 >= 0 ? mod - 1 : n - 1);
  cplx g, u, dl0;
  ent(0, dl0, g, u);
  bool u_is_a = !M.cplx_ap;   // u still equals the original interior entry a
  int i = 0;
  double r = 0.0;             // 1/|g|^2 of the previous fast step
  while (i < n - 1) {
    if (u_is_a) {
      // Fast path: keep the pivot while |g| >= a. Then |g|^2 >= a^2 > tol2 (a >= 1/(3h^2) is
      // within a factor 7 of max|T|), so no singularity test is needed. The pivots of a mode
      // settle to a fixed point, so 1/|g|^2 is refined from the previous row's: with
      // e = 1 - n2 r0, 1/n2 = r0 / (1 - e) = r0 (1 + e + e^2) + O(e^3 r0), full precision for
      // |e| < 2^-20; otherwise a division.
      // The loop-carried chain is g -> |g|^2 -> 1/|g|^2 -> g' = dd - a^2 conj(g)/|g|^2; the
      // swap test and the row's outputs branch off it.
      const double a2dd = a2;
      for (; i < fast_end; ++i) {
        const double n2 = fma(g.re, g.re, g.im * g.im);
        const double e = fma(-n2, r, 1.0);
        double rn = fma(r, fma(e, e, e), r);
        if (!(fabs(e) < 0x1p-20)) rn = rcp_pos(n2);
        if (n2 < a2) break;
        r = rn;
        const double gr = g.re * r, gi = g.im * r;   // 1/g = (gr, -gi)
        const cplx gnext = cmk(fma(-a2dd, gr, dd), a2dd * gi);
        out(i, cmk(a * gr, -a * gi), g, cmk(gr, -gi), cmk(a, 0.0), cmk(0.0, 0.0), (uint8_t)0);
        g = gnext;
      }
      if (i >= n - 1) break;
    }
    cplx lsub, gi, ui, gn, un, dln;
    ent(i, lsub, gi, ui);
    ent(i + 1, dln, gn, un);
    cplx l, dfin, dinv, dup, du2;
    uint8_t sw;
    if (!lu_step(g, u, lsub, gn, un, i == n - 2, l, dfin, dinv, dup, du2, sw)) {
      set_error(status, MDP_ERR_SINGULAR);
      return false;
    }
    if (cabs2(dfin) < tol2) { set_error(status, MDP_ERR_SINGULAR); return false; }
    out(i, l, dfin, dinv, dup, du2, sw);
    // after a kept pivot u is the original T[i+1][i+2]: a for every row but the first
    u_is_a = sw == 0;
    if (u_is_a) u = cmk(a, 0.0);
    ++i;
  }
  if (czero(g) || cabs2(g) < tol2) { set_error(status, MDP_ERR_SINGULAR); return false; }
  out(n - 1, cmk(0.0, 0.0), g, crecip(g), cmk(0.0, 0.0), cmk(0.0, 0.0), (uint8_t)0);
  return true;
}

// Chain of the full LU: raw factor rows (l, 1/d, du, du2) and swap flags.
__device__ void chain_full(const SubDesc &d, int q, double *tab, uint8_t *piv, int *status) {
  const ModeRows M = mode_rows(d, q);
  const int N = M.N, FW = d.cplx ? 8 : 4;
  const double tol2 = kSingularTolD * kSingularTolD * M.scale2();
  double *F = tab + d.fact_off + (long long)(q - 1) * N * FW;
  uint8_t *pv = piv + d.piv_off + (long long)(q - 1) * N;
  lu_chain(M, N, -1, cmk(0.0, 0.0), tol2, status,
           [&](int i, cplx l, cplx, cplx dinv, cplx du, cplx du2, uint8_t sw) {
             if (FW == 8) {
               double *r = F + (long long)i * 8;
               st2(r, l); st2(r + 2, dinv); st2(r + 4, du); st2(r + 6, du2);
             } else {
               double *r = F + (long long)i * 4;
               r[0] = l.re; r[1] = dinv.re; r[2] = du.re; r[3] = du2.re;
             }
             pv[i] = sw;
           });
}

// Chain of the condensed system (rows 0..itop, the rows above folded into the last pivot):
// raw rows i >= i0 in the sweep table: l, d, 1/d, du, du2 (complex pairs) and the swap flag;
// seg[4] = itop.
__device__ void chain_sweep(const SubDesc &d, int q, double *tab, int *status) {
  const ModeRows M = mode_rows(d, q);
  const int N = M.N;
  const double scale2 = M.scale2();
  const double tol2 = kSingularTolD * kSingularTolD * scale2, ctol2 = kCondenseTolD * kCondenseTolD * scale2;
  // top condensation: s_{N-1} = T[N-1][N-1], s_i = T[i][i] - T[i][i+1] T[i+1][i] / s_{i+1}
  const int ih = d.nhi + 1 - d.nfirst;
  int itop = N - 1;
  cplx sigma = cmk(0.0, 0.0);
  if (ih < N - 1) {
    cplx dl, sv, du;
    M.entries(N - 1, dl, sv, du);
    bool ok = cabs2(sv) > ctol2;
    for (int i = N - 2; i >= ih + 1 && ok; --i) {
      cplx li, gi, ui;
      M.entries(i, li, gi, ui);
      sv = csub(gi, cdiv(cmul(ui, li), sv));
      ok = cabs2(sv) > ctol2;
    }
    if (ok) {
      cplx li, gi, ui;
      M.entries(ih, li, gi, ui);
      itop = ih;
      sigma = cdiv(cmul(ui, li), sv);
    }
  }
  tab[d.seg_off + 5 * (q - 1) + 4] = itop;
  double *T = tab + d.fs_off + (long long)(q - 1) * d.NYf * FSW;
  lu_chain(M, itop + 1, itop, sigma, tol2, status,
           [&](int i, cplx l, cplx dg, cplx dinv, cplx du, cplx du2, uint8_t sw) {
             if (i < d.i0) return;
             double *r = T + (long long)(i - d.i0) * FSW;
             st2(r, l); st2(r + 2, dg); st2(r + 4, dinv); st2(r + 6, du); st2(r + 8, du2);
             r[22] = sw;
           });
}

__global__ void __launch_bounds__(32) k_factor_chain(const SubDesc *subs, int n_subs, int n_modes, double *tab,
                                                      uint8_t *piv, int *status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n_modes) return;
  const bool sweep = t >= n_modes;
  if (sweep) t -= n_modes;
  int si = mode_owner(subs, n_subs, t);
  if (si >= n_subs) return;
  if (sweep) chain_sweep(subs[si], t + 1, tab, status);
  else chain_full(subs[si], t + 1, tab, piv, status);
}

constexpr int kRowsThreads = 256;

// Block reduction of a real-row run: the run of rows with re[i] around row mid, from the
// largest non-real row below mid and the smallest above it.
struct RunReduce {
  int lastbad, firstbad, midreal;
  __device__ void init(int lo, int hi) { lastbad = lo - 1; firstbad = hi; midreal = 0; }
};

__global__ void __launch_bounds__(kRowsThreads) k_factor_rows(const SubDesc *subs, int n_subs, double *tab) {
  __shared__ RunReduce run;
  __shared__ double raw[(kRowsThreads + 1) * 11];
  int t = blockIdx.x;
  const int si = mode_owner(subs, n_subs, t);
  if (si >= n_subs) return;
  const SubDesc &d = subs[si];
  const int q = t + 1, tid = threadIdx.x;
  // the mode's coefficients and the 4 middle-row sines, computed once per block
  __shared__ ModeRows Ms;
  __shared__ double sines[4];
  if (tid == 0) {
    Ms = mode_rows(d, q);
    const int N2 = 2 * d.Nx;
    const int ms[4] = {d.mlo, d.mlo + 1, d.mhi - 1, d.mhi};
    for (int s_ = 0; s_ < 4; ++s_) sines[s_] = sin(M_PI * (double)((q * ms[s_]) % N2) / (double)d.Nx);
  }
  __syncthreads();
  const ModeRows &M = Ms;
  const int N = M.N;
  double *sg = tab + d.seg_off + 5 * (q - 1);
  // ---- dT/dk rows (sub, diag, super)
  double *dT = tab + d.dT_off + (long long)(q - 1) * N * 6;
  for (int i = tid; i < N; i += kRowsThreads) {
    cplx ts = cmk(M.da, 0.0), tg = cmk(M.ddd, 0.0), tu = cmk(M.da, 0.0);
    if (M.cplx_ap && i == 0) { tg = M.tp; tu = M.tm; ts = cmk(0.0, 0.0); }
    if (M.cplx_ap && i == N - 1) { tg = M.tp; ts = M.tm; tu = cmk(0.0, 0.0); }
    if (i == 0) ts = cmk(0.0, 0.0);
    if (i == N - 1) tu = cmk(0.0, 0.0);
    double *r = dT + 6 * i;
    r[0] = ts.re; r[1] = ts.im; r[2] = tg.re; r[3] = tg.im; r[4] = tu.re; r[5] = tu.im;
  }
  // ---- factor rows: (l, 1/d, du, du2) -> (l, 1/d, du/d, du2/d); real run around N/2
  if (d.cplx) {
    double *F = tab + d.fact_off + (long long)(q - 1) * N * 8;
    const int mid = N / 2;
    if (tid == 0) run.init(0, N);
    __syncthreads();
    for (int i = tid; i < N; i += kRowsThreads) {
      double *r = F + (long long)i * 8;
      const cplx l = ld2(r), dinv = ld2(r + 2);
      const cplx u1 = cmul(ld2(r + 4), dinv), u2 = cmul(ld2(r + 6), dinv);
      st2(r + 4, u1);
      st2(r + 6, u2);
      const bool re = tiny_im(l) && tiny_im(dinv) && tiny_im(u1) && tiny_im(u2);
      if (!re && i < mid) atomicMax(&run.lastbad, i);
      if (!re && i > mid) atomicMin(&run.firstbad, i);
      if (re && i == mid) run.midreal = 1;
    }
    __syncthreads();
    const int rlo = run.midreal ? run.lastbad + 1 : mid, rhi = run.midreal ? run.firstbad : mid;
    for (int i = tid; i < N; i += kRowsThreads)
      if (i >= rlo && i < rhi)
        for (int w = 0; w < 4; ++w) F[(long long)i * 8 + 2 * w + 1] = 0.0;
    if (tid == 0) { sg[0] = rlo; sg[1] = rhi; }
    __syncthreads();
  } else {
    double *F = tab + d.fact_off + (long long)(q - 1) * N * 4;
    for (int i = tid; i < N; i += kRowsThreads) {
      double *r = F + (long long)i * 4;
      const double dinv = r[1];
      r[2] *= dinv;
      r[3] *= dinv;
    }
    if (tid == 0) { sg[0] = 0; sg[1] = N; }
  }
  // ---- sweep rows i0 .. itop from the raw rows, in chunks of kRowsThreads rows
  const int itop = (int)sg[4], i0 = d.i0;
  const int mid = (i0 + itop) / 2;
  double *T = tab + d.fs_off + (long long)(q - 1) * d.NYf * FSW;
  if (tid == 0) run.init(i0, itop + 1);
  __syncthreads();
  for (int c0 = i0; c0 <= itop; c0 += kRowsThreads) {
    const int nr = min(kRowsThreads + 1, itop + 1 - c0);   // raw rows c0 .. c0 + nr - 1
    for (int k = tid; k < nr * 11; k += kRowsThreads) {
      const int rr = k / 11, w = k % 11;
      raw[rr * 11 + w] = T[(long long)(c0 + rr - i0) * FSW + (w < 10 ? w : 22)];
    }
    __syncthreads();
    const int i = c0 + tid;
    if (tid < kRowsThreads && i <= itop) {
      const double *rw = raw + tid * 11;
      const bool last = i == itop;
      const cplx l = last ? cmk(0.0, 0.0) : cmk(rw[0], rw[1]);
      const cplx di = cmk(rw[2], rw[3]), dinv = cmk(rw[4], rw[5]);
      const cplx du = cmk(rw[6], rw[7]), du2 = cmk(rw[8], rw[9]);
      const cplx dni = last ? cmk(0.0, 0.0) : cmk(rw[11 + 4], rw[11 + 5]);
      cplx v[11];
      v[0] = cmul(cmul(l, di), dni);
      v[1] = cmul(di, dni);
      v[2] = cmul(l, dni);
      v[3] = dinv;
      v[4] = dni;
      for (int s_ = 0; s_ < 4; ++s_) v[5 + s_] = cscale(sines[s_], dni);
      v[9] = last ? cmk(0.0, 0.0) : cmul(du, dinv);
      v[10] = i + 2 <= itop ? cmul(du2, dinv) : cmk(0.0, 0.0);
      double *row = T + (long long)(i - i0) * FSW;
      bool re = true;
      for (int w = 0; w < 11; ++w) {
        row[2 * w] = v[w].re;
        row[2 * w + 1] = v[w].im;
        re = re && tiny_im(v[w]);
      }
      row[22] = rw[10];
      row[23] = 0.0;
      if (!re && i < mid) atomicMax(&run.lastbad, i);
      if (!re && i > mid) atomicMin(&run.firstbad, i);
      if (re && i == mid) run.midreal = 1;
    }
    __syncthreads();
  }
  const int flo = run.midreal ? run.lastbad + 1 : mid, fhi = run.midreal ? run.firstbad : mid;
  for (int i = i0 + tid; i <= itop; i += kRowsThreads)
    if (i >= flo && i < fhi) {
      double *row = T + (long long)(i - i0) * FSW;
      for (int w = 0; w < 11; ++w) row[2 * w + 1] = 0.0;
    }
  if (tid == 0) { sg[2] = flo; sg[3] = fhi; }
}

__global__ void k_probe_rcp(const double *x, double *y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = rcp_pos(x[i]);
}

}  // namespace

// The chains: one thread each, warps spread one per block so that they do not share an SM's
// FP64 unit while there are fewer warps than SMs. The row kernel: one block per mode.
cudaError_t launch_factor(const mdp_plan *p, int *status, cudaStream_t st) {
  return launch_factor_to(p, p->d_subs, p->d_tables, p->d_piv, status, st);
}

cudaError_t launch_factor_to(const mdp_plan *p, const SubDesc *ds, double *tab, uint8_t *piv, int *status,
                             cudaStream_t st) {
  int n_modes = 0;
  for (size_t i = 0; i < p->subs.size(); ++i)
    if (p->subs[i].d.leader == (int)i) n_modes += p->subs[i].d.Nq;
  const int threads = 2 * n_modes;
  k_factor_chain<<<(threads + 31) / 32, 32, 0, st>>>(ds, (int)p->subs.size(), n_modes, tab, piv, status);
  k_factor_rows<<<n_modes, kRowsThreads, 0, st>>>(ds, (int)p->subs.size(), tab);
  return cudaGetLastError();
}

}  // namespace mdp

// The reciprocal of the factorisation chains on device arrays (test probe, include/mdp_probe.h).
extern "C" mdp_status mdp_probe_rcp(const double *x, double *y, int n, void *cuda_stream) {
  if (n < 0 || (n > 0 && (!x || !y))) return MDP_ERR_ARG;
  if (n == 0) return MDP_OK;
  mdp::k_probe_rcp<<<(n + 255) / 256, 256, 0, (cudaStream_t)cuda_stream>>>(x, y, n);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_ERR_CUDA;
}
