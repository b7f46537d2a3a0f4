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
// factor_mode, build_fs_mode). Here one thread streams one mode's rows with O(1) state, so
// no per-mode scratch is needed: thread t < M factors mode t fully, thread M + t builds the
// sweep table of mode t (M = number of modes of all subdomains).
#include "kernels_common.cuh"

namespace mdp {
namespace {

constexpr double kSingularTolD = 1e-13;   // pivot below this x max|T| -> singular
constexpr double kCondenseTolD = 1e-8;    // Schur complement below this x max|T|: keep all rows

__device__ __forceinline__ double cabs2(cplx a) { return fma(a.re, a.re, a.im * a.im); }
__device__ __forceinline__ cplx cscale(double s, cplx a) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ bool czero(cplx a) { return a.re == 0.0 && a.im == 0.0; }
// 1/b and a/b through one real reciprocal of |b|^2 (the magnitudes here are O(1/h^2), far from
// overflow and underflow)
__device__ __forceinline__ cplx crecip(cplx b) {
  const double r = 1.0 / cabs2(b);
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
  const double alpha = (1.0 + k2 * h2 / 24.0 + lam / 24.0) / h2;
  const double beta = k * (1.0 + k2 * h2 / 8.0 + lam / 8.0) / h;           // imaginary part
  const double dalpha = k / 12.0;
  const double dbeta = (1.0 + 3.0 * k2 * h2 / 8.0 + lam / 8.0) / h;        // imaginary part
  m.cp = cmk(alpha, 0.5 * beta);
  m.cm = cmk(-alpha, 0.5 * beta);
  m.tp = cmk(dalpha, 0.5 * dbeta);
  m.tm = cmk(-dalpha, 0.5 * dbeta);
  return m;
}

// One step of the banded LU with partial pivoting, streamed: on entry (g, u) are the current
// diagonal and super-diagonal of row i, (lsub, gn, un) the original T[i+1][i], T[i+1][i+1],
// T[i+1][i+2]. On exit (l, dfin, dup, du2, sw) are row i's multiplier, pivot, first and second
// super-diagonal of U and swap flag, and (g, u) hold row i+1. last2: i == n-2 (no du2 fill-in).
// Returns false on a zero pivot.
__device__ __forceinline__ bool lu_step(cplx &g, cplx &u, cplx lsub, cplx gn, cplx un, bool last2, cplx &l,
                                        cplx &dfin, cplx &dinv, cplx &dup, cplx &du2, uint8_t &sw) {
  if (cabs2(g) >= cabs2(lsub)) {
    if (czero(g)) return false;
    dinv = crecip(g);
    const cplx f = cmul(lsub, dinv);
    l = f; dfin = g; dup = u; du2 = cmk(0.0, 0.0); sw = 0;
    g = csub(gn, cmul(f, u));
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

// Full LU of T_q: factor rows, swap flags, dT/dk rows, seg[0..1] (real-row run).
__device__ void factor_full(const SubDesc &d, int q, double *tab, uint8_t *piv, int *status) {
  const ModeRows M = mode_rows(d, q);
  const int N = M.N, FW = d.cplx ? 8 : 4;
  const double tol2 = kSingularTolD * kSingularTolD * M.scale2();
  double *F = tab + d.fact_off + (long long)(q - 1) * N * FW;
  double *dT = tab + d.dT_off + (long long)(q - 1) * N * 6;
  uint8_t *pv = piv + d.piv_off + (long long)(q - 1) * N;
  // dT/dk rows: (sub, diag, super)
  for (int i = 0; i < N; ++i) {
    cplx ts = cmk(M.da, 0.0), tg = cmk(M.ddd, 0.0), tu = cmk(M.da, 0.0);
    if (M.cplx_ap && i == 0) { tg = M.tp; tu = M.tm; ts = cmk(0.0, 0.0); }
    if (M.cplx_ap && i == N - 1) { tg = M.tp; ts = M.tm; tu = cmk(0.0, 0.0); }
    if (i == 0) ts = cmk(0.0, 0.0);
    if (i == N - 1) tu = cmk(0.0, 0.0);
    double *t = dT + 6 * i;
    t[0] = ts.re; t[1] = ts.im; t[2] = tg.re; t[3] = tg.im; t[4] = tu.re; t[5] = tu.im;
  }
  cplx g, u, dl0;
  M.entries(0, dl0, g, u);
  const int mid = N / 2;
  int lastbad = -1, rlo = mid, rhi = mid;
  bool inrun = false;
  for (int i = 0; i < N; ++i) {
    cplx l = cmk(0.0, 0.0), dfin, dinv, dup = cmk(0.0, 0.0), du2 = cmk(0.0, 0.0);
    uint8_t sw = 0;
    if (i < N - 1) {
      cplx lsub, gi, ui, gn, un, dln;
      M.entries(i, lsub, gi, ui);
      M.entries(i + 1, dln, gn, un);
      if (!lu_step(g, u, lsub, gn, un, i == N - 2, l, dfin, dinv, dup, du2, sw)) {
        set_error(status, MDP_ERR_SINGULAR);
        return;
      }
    } else {
      if (czero(g)) { set_error(status, MDP_ERR_SINGULAR); return; }
      dfin = g;
      dinv = crecip(g);
    }
    if (cabs2(dfin) < tol2) { set_error(status, MDP_ERR_SINGULAR); return; }
    const cplx u1 = i < N - 1 ? cmul(dup, dinv) : cmk(0.0, 0.0);
    const cplx u2 = i < N - 2 ? cmul(du2, dinv) : cmk(0.0, 0.0);
    if (i >= N - 1) l = cmk(0.0, 0.0);
    if (FW == 8) {
      double *r = F + (long long)i * 8;
      r[0] = l.re; r[1] = l.im; r[2] = dinv.re; r[3] = dinv.im; r[4] = u1.re; r[5] = u1.im; r[6] = u2.re; r[7] = u2.im;
      const bool re = tiny_im(l) && tiny_im(dinv) && tiny_im(u1) && tiny_im(u2);
      if (i < mid && !re) lastbad = i;
      if (i == mid) {
        if (re) { rlo = lastbad + 1; inrun = true; }
      } else if (i > mid && inrun && !re) {
        rhi = i;
        inrun = false;
      }
    } else {
      double *r = F + (long long)i * 4;
      r[0] = l.re; r[1] = dinv.re; r[2] = u1.re; r[3] = u2.re;
    }
    pv[i] = sw;
  }
  if (inrun) rhi = N;
  if (FW == 8) {
    for (int i = rlo; i < rhi; ++i)
      for (int w = 0; w < 4; ++w) F[(long long)i * 8 + 2 * w + 1] = 0.0;
  } else {
    rlo = 0; rhi = N;
  }
  double *sg = tab + d.seg_off + 5 * (q - 1);
  sg[0] = rlo;
  sg[1] = rhi;
}

// Condensed, pivot-scaled forward-sweep table of mode q and seg[2..4] (real run, itop).
// Row layout (complex pairs): m = l d_i/d_{i+1}, d_i/d_{i+1}, l/d_{i+1}, 1/d_i, 1/d_{i+1},
// c0..c3 = sin(pi q m_s/Nx)/d_{i+1} (m_s = mlo, mlo+1, mhi-1, mhi), du_i/d_i, du2_i/d_i, then the
// swap flag and a pad.
__device__ void factor_sweep(const SubDesc &d, int q, double *tab, int *status) {
  const ModeRows M = mode_rows(d, q);
  const int N = M.N;
  const double scale2 = M.scale2();
  const double tol2 = kSingularTolD * kSingularTolD * scale2, ctol2 = kCondenseTolD * kCondenseTolD * scale2;
  // (1) top condensation
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
  const int n = itop + 1;
  auto entries_c = [&](int i, cplx &dl, cplx &dg, cplx &du) {
    M.entries(i, dl, dg, du);
    if (i == itop) dg = csub(dg, sigma);
  };
  // (2) condensed LU, emitting sweep row i once d_{i+1} is final
  const int N2 = 2 * d.Nx;
  const int ms[4] = {d.mlo, d.mlo + 1, d.mhi - 1, d.mhi};
  double sines[4];
  for (int s_ = 0; s_ < 4; ++s_) sines[s_] = sin(M_PI * (double)((q * ms[s_]) % N2) / (double)d.Nx);
  double *T = tab + d.fs_off + (long long)(q - 1) * d.NYf * FSW;
  const int mid = (d.i0 + itop) / 2;
  int lastbad = d.i0 - 1, flo = mid, fhi = mid;
  bool inrun = false;
  // row i of the sweep table from its LU row (l, d_i, 1/d_i, du, du2) and 1/d_{i+1}
  auto emit = [&](int i, cplx l, cplx di, cplx dinv, cplx dni, cplx dup, cplx du2, uint8_t sw, bool last) {
    if (i < d.i0) return;
    if (last) { l = cmk(0.0, 0.0); dni = cmk(0.0, 0.0); }
    cplx v[11];
    v[0] = cmul(cmul(l, di), dni);
    v[1] = cmul(di, dni);
    v[2] = cmul(l, dni);
    v[3] = dinv;
    v[4] = dni;
    for (int s_ = 0; s_ < 4; ++s_) v[5 + s_] = cscale(sines[s_], dni);
    v[9] = last ? cmk(0.0, 0.0) : cmul(dup, dinv);
    v[10] = i + 2 <= itop ? cmul(du2, dinv) : cmk(0.0, 0.0);
    double *row = T + (long long)(i - d.i0) * FSW;
    bool re = true;
    for (int w = 0; w < 11; ++w) {
      row[2 * w] = v[w].re;
      row[2 * w + 1] = v[w].im;
      re = re && tiny_im(v[w]);
    }
    row[22] = sw;
    row[23] = 0.0;
    if (i < mid && !re) lastbad = i;
    if (i == mid) {
      if (re) { flo = lastbad + 1; inrun = true; }
    } else if (i > mid && inrun && !re) {
      fhi = i;
      inrun = false;
    }
  };
  cplx g, u, dl0;
  entries_c(0, dl0, g, u);
  // pending row (its pivot d_i is final; d_{i+1} is not yet)
  cplx pl = cmk(0.0, 0.0), pd = cmk(0.0, 0.0), pdi = cmk(0.0, 0.0), pdu = cmk(0.0, 0.0), pdu2 = cmk(0.0, 0.0);
  uint8_t psw = 0;
  for (int i = 0; i < n; ++i) {
    cplx l = cmk(0.0, 0.0), dfin, dinv, dup = cmk(0.0, 0.0), du2 = cmk(0.0, 0.0);
    uint8_t sw = 0;
    if (i < n - 1) {
      cplx lsub, gi, ui, gn, un, dln;
      entries_c(i, lsub, gi, ui);
      entries_c(i + 1, dln, gn, un);
      if (!lu_step(g, u, lsub, gn, un, i == n - 2, l, dfin, dinv, dup, du2, sw)) {
        set_error(status, MDP_ERR_SINGULAR);
        return;
      }
    } else {
      if (czero(g)) { set_error(status, MDP_ERR_SINGULAR); return; }
      dfin = g;
      dinv = crecip(g);
    }
    if (cabs2(dfin) < tol2) { set_error(status, MDP_ERR_SINGULAR); return; }
    if (i > 0) emit(i - 1, pl, pd, pdi, dinv, pdu, pdu2, psw, false);
    pl = l; pd = dfin; pdi = dinv; pdu = dup; pdu2 = du2; psw = sw;
  }
  emit(itop, pl, pd, pdi, cmk(0.0, 0.0), pdu, pdu2, psw, true);
  if (inrun) fhi = itop + 1;
  for (int i = flo; i < fhi; ++i) {
    double *row = T + (long long)(i - d.i0) * FSW;
    for (int w = 0; w < 11; ++w) row[2 * w + 1] = 0.0;
  }
  double *sg = tab + d.seg_off + 5 * (q - 1);
  sg[2] = flo;
  sg[3] = fhi;
  sg[4] = itop;
}

__global__ void __launch_bounds__(32) k_factor(const SubDesc *subs, int n_subs, int n_modes, double *tab,
                                                uint8_t *piv, int *status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n_modes) return;
  const bool sweep = t >= n_modes;
  if (sweep) t -= n_modes;
  int si = 0;
  while (si < n_subs && t >= subs[si].Nq) { t -= subs[si].Nq; ++si; }
  if (si >= n_subs) return;
  if (sweep) factor_sweep(subs[si], t + 1, tab, status);
  else factor_full(subs[si], t + 1, tab, piv, status);
}

}  // namespace

// Each thread is one long dependent chain of FP64 operations and an SM retires 2 FP64 lanes per
// clock, so the warps are spread one per block (one per SM while there are fewer warps than SMs)
// instead of packed four to an SM.
cudaError_t launch_factor(const mdp_plan *p, int *status, cudaStream_t st) {
  int n_modes = 0;
  for (auto &hs : p->subs) n_modes += hs.d.Nq;
  const int threads = 2 * n_modes;
  k_factor<<<(threads + 31) / 32, 32, 0, st>>>(p->d_subs, (int)p->subs.size(), n_modes, p->d_tables, p->d_piv,
                                                status);
  return cudaGetLastError();
}

}  // namespace mdp
