// Host side of the plan: grid sets and gamma (Section 3.2.2), the per-mode tridiagonal
// systems of the discrete AP along y after the sine transform along x (Section 3.2.1),
// their pivoted LU factors, sine tables and the batch schedule.
//
// Compiled with -ffp-contract=off so that the floating-point decisions that pick integer
// sets (M+ membership, side ownership) are the plain IEEE operations x = ax0 + m*h etc.
#include "mdp_internal.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <atomic>
#include <cstring>
#include <thread>

namespace mdp {

using cd = std::complex<double>;

static const double kTieTol = 1e-9;       // side-ownership ties within 1e-9*h
static const double kSingularTol = 1e-13; // pivot below this x max|T| -> singular

const char *fam_name(int f) {
  static const char *names[NFAM] = {"k_extend", "k_residual", "k_fwd_rows", "k_tri", "k_inv_rows", "k_inv_cols",
                                    "k_adj_rows", "k_adj_tri", "k_adj_ring_rows", "k_adj_ring_cols", "k_adj_gamma",
                                    "k_inv_rec", "k_adj_cols", "k_inv_cols_tc", "k_adj_ring_cols_tc"};
  return (f >= 0 && f < NFAM) ? names[f] : "?";
}

// ---------------------------------------------------------------- geometry
static mdp_status geometry(const mdp_subdomain &in, HostSub &hs, unsigned flags, int fft_block_points) {
  SubDesc &d = hs.d;
  std::memset(&d, 0, sizeof d);
  if (in.nx < 9 || in.ny < 9 || !(in.h > 0) || !(in.k > 0) || in.n_modes < 1 ||
      (in.ap_bc != MDP_AP_DIRICHLET4 && in.ap_bc != MDP_AP_DIRX_SOMMY && in.ap_bc != MDP_AP_DIRX_SOMMY_PAPER) ||
      !(in.x1 > in.x0) ||
      !(in.y1 > in.y0) || !std::isfinite(in.k))
    return MDP_ERR_ARG;
  d.nx = in.nx; d.ny = in.ny; d.Nx = in.nx - 1; d.Nq = d.Nx - 1;
  d.h = in.h; d.k = in.k;
  d.x0 = in.x0; d.x1 = in.x1; d.y0 = in.y0; d.y1 = in.y1; d.ax0 = in.ax0; d.ay0 = in.ay0;
  d.ap_bc = in.ap_bc; d.cplx = in.ap_bc != MDP_AP_DIRICHLET4;
  d.n_modes = in.n_modes; d.n_cols = 8 * in.n_modes;
  // M+ = M0 nodes strictly inside the open subdomain: an interval along each axis.
  int mlo = -1, mhi = -1, nlo = -1, nhi = -1;
  for (int m = 1; m <= in.nx - 2; ++m) {
    double x = in.ax0 + (double)m * in.h;
    if (in.x0 < x && x < in.x1) { if (mlo < 0) mlo = m; mhi = m; }
  }
  for (int n = 1; n <= in.ny - 2; ++n) {
    double y = in.ay0 + (double)n * in.h;
    if (in.y0 < y && y < in.y1) { if (nlo < 0) nlo = n; nhi = n; }
  }
  if (mlo < 0 || nlo < 0) return MDP_ERR_ARG;
  d.mlo = mlo; d.mhi = mhi; d.nlo = nlo; d.nhi = nhi;
  d.Px = mhi - mlo + 1; d.Py = nhi - nlo + 1;
  // gamma must stay one node inside the AP boundary, and the ring must not degenerate
  if (mlo < 2 || mhi > in.nx - 3 || nlo < 2 || nhi > in.ny - 3 || d.Px < 5 || d.Py < 5) return MDP_ERR_ARG;
  d.G = 4 * (d.Px + d.Py);
  d.R = 4 * d.Px + 4 * (d.Py - 4);
  // centred along x: the ring pairs m with Nx - m (sin(pi q (Nx-m)/Nx) = (-1)^(q+1) sin(pi q m/Nx))
  d.xsym = (mlo + mhi == d.Nx) && (d.Nx % 2 == 0);
  d.Ph = d.xsym ? d.Nx / 2 - mlo + 1 : 0;
  d.R2 = d.xsym ? 8 * d.Ph + 4 * (d.Py - 4) : d.R;  // (sum, difference) per pair unit
  d.nrec = -1;
  d.rows_fft = !(flags & MDP_PLAN_DIRECT_ROWS) && (d.Nx & (d.Nx - 1)) == 0 && 2 * d.Nx <= FFT_POINTS && d.Nx >= 8;
  d.fpb = d.rows_fft ? std::max(1, fft_block_points / (2 * d.Nx)) : 0;
  // gamma columns on the tensor cores: exact integer accumulation needs at most 1024 modes per
  // output (a parity half of Nq on centred subdomains); MDP_PLAN_FP64_COLS (or the environment
  // MDP_TC_COLS=0) keeps the FP64 sums
  {
    const char *tc = std::getenv("MDP_TC_COLS");
    const bool on = !(flags & MDP_PLAN_FP64_COLS) && !(tc && tc[0] == '0' && tc[1] == 0);
    d.tc_cols = on && (d.xsym ? d.Nq <= 2047 : d.Nq <= 1023);
  }
  d.nfirst = d.cplx ? 0 : 1;
  d.Nt = d.cplx ? in.ny : in.ny - 2;
  d.i0 = (nlo - 1) - d.nfirst;
  d.NYf = d.Nt - d.i0;
  // 9-point coefficients (Eq. FD_scheme): centre, edge, corner, and their k-derivatives
  const double h2 = in.h * in.h, k2 = in.k * in.k;
  d.c2 = 1.0 / (6.0 * h2);
  d.c1 = 1.0 / h2 - 2.0 / (6.0 * h2) + k2 / 12.0;
  d.c0 = -4.0 / h2 + 4.0 / (6.0 * h2) + 8.0 * k2 / 12.0;
  d.dc1 = in.k / 6.0;
  d.dc0 = 8.0 * in.k / 6.0;
  // gamma nodes in row-major order with side ownership
  hs.gamma_nm.clear(); hs.owner.clear(); hs.rho.clear(); hs.s.clear(); hs.L.clear();
  const double lx = in.x1 - in.x0, ly = in.y1 - in.y0;
  for (int n = nlo - 1; n <= nhi + 1; ++n) {
    const bool full = (n <= nlo || n >= nhi);
    for (int m = mlo - 1; m <= mhi + 1; ++m) {
      if (!full && !(m <= mlo || m >= mhi)) continue;
      const double gx = in.ax0 + (double)m * in.h, gy = in.ay0 + (double)n * in.h;
      const double rhos[4] = {in.y0 - gy, gy - in.y1, in.x0 - gx, gx - in.x1};
      double dmin = std::fabs(rhos[0]);
      for (int i = 1; i < 4; ++i) dmin = std::min(dmin, std::fabs(rhos[i]));
      const double lim = dmin + kTieTol * in.h;
      int own = 0;
      while (!(std::fabs(rhos[own]) <= lim)) ++own;
      hs.gamma_nm.push_back(n);
      hs.gamma_nm.push_back(m);
      hs.owner.push_back(own + 1);
      hs.rho.push_back(rhos[own]);
      hs.s.push_back(own <= 1 ? 2.0 * (gx - in.x0) / lx - 1.0 : 2.0 * (gy - in.y0) / ly - 1.0);
      hs.L.push_back(own <= 1 ? lx : ly);
    }
  }
  if ((int)hs.owner.size() != d.G) return MDP_ERR_ARG;
  return MDP_OK;
}

// ---------------------------------------------------------------- tridiagonal factors
// T_q: the discrete AP restricted to sine mode q along x (lambda_q = -4 sin^2(pi q/(2Nx)),
// the eigenvalue of the undivided second difference with zero ends):
//   interior rows  a u_{n-1} + d u_n + a u_{n+1},
//     a = 1/h^2 + lambda/(6h^2) + k^2/12,  d = -2a + lambda/h^2 + k^2 + k^2 lambda/12;
//   Sommerfeld rows (scaled by 1/h): alpha (u_N - u_{N-1}) + beta (u_N + u_{N-1})/2 = 0 with
//     alpha = (1 + k^2h^2/24 + lambda/24)/h^2,  beta = i k (1 + k^2h^2/8 + lambda/8)/h,
//   and the mirror image at n = 0; as printed (MDP_AP_DIRX_SOMMY_PAPER)
//     alpha = (1 - k^2h^2/24 - lambda/6)/h^2,   beta = i k (1 + k^2h^2/8 + lambda/2)/h.
// Factorisation: Gaussian elimination with partial pivoting on the band (row swaps create
// one extra super-diagonal), the textbook algorithm for banded LU.
// The tridiagonal T_q of sine mode q (rows 0..Nt-1) and, when dT != nullptr, its k-derivative
// rows (sub, diag, super; complex). dl[i] = T[i+1][i], dg[i] = T[i][i], du[i] = T[i][i+1].
static void mode_matrix(const SubDesc &d, int q, cd *dl, cd *dg, cd *du, double *dT) {
  const int N = d.Nt;
  const double h = d.h, h2 = h * h, k = d.k, k2 = k * k;
  const double sq = std::sin(M_PI * q / (2.0 * d.Nx));
  const double lam = -4.0 * sq * sq;
  const double a = 1.0 / h2 + lam / (6.0 * h2) + k2 / 12.0;
  const double dd = -2.0 * a + lam / h2 + k2 + k2 * lam / 12.0;
  const double da = k / 6.0;
  const double ddd = -2.0 * da + 2.0 * k + 2.0 * k * lam / 12.0;
  const bool paper = d.ap_bc == MDP_AP_DIRX_SOMMY_PAPER;
  const cd alpha(paper ? (1.0 - k2 * h2 / 24.0 - lam / 6.0) / h2 : (1.0 + k2 * h2 / 24.0 + lam / 24.0) / h2, 0.0);
  const cd beta(0.0, k * (1.0 + k2 * h2 / 8.0 + lam / (paper ? 2.0 : 8.0)) / h);
  const cd dalpha(paper ? -k / 12.0 : k / 12.0, 0.0);
  const cd dbeta(0.0, (1.0 + 3.0 * k2 * h2 / 8.0 + lam / (paper ? 2.0 : 8.0)) / h);
  for (int i = 0; i < N; ++i) {
    dl[i] = a; dg[i] = dd; du[i] = a;
    cd tsub = da, tdg = ddd, tsup = da;
    if (d.cplx && i == 0) { dg[i] = alpha + 0.5 * beta; du[i] = -alpha + 0.5 * beta; tdg = dalpha + 0.5 * dbeta; tsup = -dalpha + 0.5 * dbeta; tsub = 0.0; }
    if (d.cplx && i == N - 1) { dg[i] = alpha + 0.5 * beta; tdg = dalpha + 0.5 * dbeta; tsub = -dalpha + 0.5 * dbeta; tsup = 0.0; }
    if (i == 0) tsub = 0.0;
    if (i == N - 1) tsup = 0.0;
    if (dT) {
      dT[i * 6 + 0] = tsub.real(); dT[i * 6 + 1] = tsub.imag();
      dT[i * 6 + 2] = tdg.real();  dT[i * 6 + 3] = tdg.imag();
      dT[i * 6 + 4] = tsup.real(); dT[i * 6 + 5] = tsup.imag();
    }
  }
  // the top Sommerfeld row's sub-diagonal entry is T[N-1][N-2] = dl[N-2]
  if (d.cplx) dl[N - 2] = -alpha + 0.5 * beta;
}

// Banded LU with partial pivoting of rows 0..N-1 in place: on return dl holds the multipliers,
// dg the pivots, du / du2 the first / second super-diagonal of U, pv the row swaps.
static bool band_lu(int N, cd *dl, cd *dg, cd *du, cd *du2, uint8_t *pv) {
  for (int i = 0; i < N; ++i) du2[i] = 0.0;
  for (int i = 0; i < N - 1; ++i) {
    if (std::abs(dg[i]) >= std::abs(dl[i])) {
      if (dg[i] == 0.0) return false;
      const cd f = dl[i] / dg[i];
      dl[i] = f;
      dg[i + 1] -= f * du[i];
      du2[i] = 0.0;
      pv[i] = 0;
    } else {
      const cd f = dg[i] / dl[i];
      dg[i] = dl[i];
      dl[i] = f;
      const cd tmp = du[i];
      du[i] = dg[i + 1];
      dg[i + 1] = tmp - f * dg[i + 1];
      if (i < N - 2) { du2[i] = du[i + 1]; du[i + 1] = -f * du[i + 1]; }
      pv[i] = 1;
    }
  }
  pv[N - 1] = 0;
  return true;
}

static bool tiny_imag(cd v) { return std::fabs(v.imag()) <= 0x1p-60 * std::abs(v); }

// The projection's forward-sweep table (rows i0 .. Nt-1 of each mode, FSW doubles per row).
// (1) Top condensation: rows above itop = nhi + 1 - nfirst carry zero right-hand side in the
//     projection, so they are eliminated into the last pivot by their Schur complement
//     T[itop][itop] -= T[itop][itop+1] T[itop+1][itop] / s_{itop+1}, s computed from the top row
//     down (s_{N-1} = T[N-1][N-1], s_i = T[i][i] - T[i][i+1] T[i+1][i] / s_{i+1}); the condensed
//     system (rows 0..itop) is factored with the same pivoted band LU. A mode whose s is tiny
//     relative to the matrix (a resonance of the rows above) keeps all rows (itop = Nt-1).
// (2) Pivot-scaled sweep: with y~_i = y_i / d_i stored, the back substitution is
//     x_i = y~_i - (du_i/d_i) x_{i+1} - (du2_i/d_i) x_{i+2}; the forward sweep carries
//     c~ = cur / d at each position: unswapped step c~' = g^_{i+1} - m_i c~ with
//     m_i = l_i d_i / d_{i+1}, g^ = g / d_{i+1}; swapped step y~_i = g / d_i and
//     c~' = (d_i / d_{i+1}) c~ - (l_i / d_{i+1}) g.
// Row layout (complex pairs): m, p = d_i/d_{i+1}, mq = l_i/d_{i+1}, qd = 1/d_i, sc = 1/d_{i+1},
// c0..c3 = sc * sin(pi q m_s / Nx) for the ring columns m_s = mlo, mlo+1, mhi-1, mhi, u1, u2,
// then the swap flag and a pad. seg[2], seg[3]: rows with real entries [frlo, frhi); seg[4] = itop.
static mdp_status build_fs_mode(HostSub &hs, int q) {
  SubDesc &d = hs.d;
  const int N = d.Nt, R = d.NYf;
  std::vector<cd> dl(N), dg(N), du(N), du2(N), T_dl(N), T_dg(N), T_du(N);
  std::vector<uint8_t> pv(N);
  const int ih = d.nhi + 1 - d.nfirst;
  {
    mode_matrix(d, q, T_dl.data(), T_dg.data(), T_du.data(), nullptr);
    double scale = 0.0;
    for (int i = 0; i < N; ++i) scale = std::max({scale, std::abs(T_dg[i]), std::abs(T_du[i]), std::abs(T_dl[i])});
    int itop = N - 1;
    cd sigma = 0.0;
    if (ih < N - 1) {
      cd sv = T_dg[N - 1];
      bool ok = std::abs(sv) > 1e-8 * scale;
      for (int i = N - 2; i >= ih + 1 && ok; --i) {
        sv = T_dg[i] - T_du[i] * T_dl[i] / sv;
        ok = std::abs(sv) > 1e-8 * scale;
      }
      if (ok) { itop = ih; sigma = T_du[ih] * T_dl[ih] / sv; }
    }
    const int n = itop + 1;
    for (int i = 0; i < n; ++i) { dl[i] = T_dl[i]; dg[i] = T_dg[i]; du[i] = T_du[i]; }
    dg[itop] -= sigma;
    if (!band_lu(n, dl.data(), dg.data(), du.data(), du2.data(), pv.data())) return MDP_ERR_SINGULAR;
    for (int i = 0; i < n; ++i)
      if (std::abs(dg[i]) < kSingularTol * scale) return MDP_ERR_SINGULAR;
    const int N2 = 2 * d.Nx;
    const int ms[4] = {d.mlo, d.mlo + 1, d.mhi - 1, d.mhi};
    double sines[4];
    for (int s_ = 0; s_ < 4; ++s_) sines[s_] = std::sin(M_PI * (double)((q * ms[s_]) % N2) / (double)d.Nx);
    double *F = hs.fs + (size_t)(q - 1) * R * FSW;
    std::vector<uint8_t> isreal(R, 1);
    for (int i = d.i0; i <= itop; ++i) {
      double *row = F + (size_t)(i - d.i0) * FSW;
      const cd dinv = 1.0 / dg[i];
      const bool last = i == itop;
      const cd dnext_inv = last ? cd(0.0) : 1.0 / dg[i + 1];
      const cd l = last ? cd(0.0) : dl[i];
      const cd vals[11] = {l * dg[i] * dnext_inv, dg[i] * dnext_inv, l * dnext_inv, dinv, dnext_inv,
                           dnext_inv * sines[0], dnext_inv * sines[1], dnext_inv * sines[2], dnext_inv * sines[3],
                           last ? cd(0.0) : du[i] * dinv, i + 2 <= itop ? du2[i] * dinv : cd(0.0)};
      bool re = true;
      for (int w = 0; w < 11; ++w) {
        row[2 * w] = vals[w].real();
        row[2 * w + 1] = vals[w].imag();
        re = re && tiny_imag(vals[w]);
      }
      row[22] = pv[i];
      isreal[i - d.i0] = re;
    }
    // real rows: the longest run containing the middle of the swept range
    const int mid = (d.i0 + itop) / 2 - d.i0;
    int flo = mid, fhi = mid;
    if (isreal[mid]) {
      flo = mid; fhi = mid + 1;
      while (flo > 0 && isreal[flo - 1]) --flo;
      while (fhi < itop - d.i0 + 1 && isreal[fhi]) ++fhi;
      for (int r = flo; r < fhi; ++r)
        for (int w = 0; w < 11; ++w) F[(size_t)r * FSW + 2 * w + 1] = 0.0;
    }
    hs.seg[(size_t)(q - 1) * 5 + 2] = flo + d.i0;
    hs.seg[(size_t)(q - 1) * 5 + 3] = fhi + d.i0;
    hs.seg[(size_t)(q - 1) * 5 + 4] = itop;
  }
  return MDP_OK;
}


// Factor mode q of subdomain hs (tables sized by prepare_tables): the full pivoted LU of T_q
// (factor table, dT/dk rows, real-row run) and the condensed, pivot-scaled forward-sweep table.
static mdp_status factor_mode(HostSub &hs, int q) {
  SubDesc &d = hs.d;
  const int N = d.Nt, FW = d.cplx ? 8 : 4;
  std::vector<cd> dl(N), dg(N), du(N), du2(N);
  mode_matrix(d, q, dl.data(), dg.data(), du.data(), hs.dT + (size_t)(q - 1) * N * 6);
  double scale = 0.0;
  for (int i = 0; i < N; ++i) scale = std::max({scale, std::abs(dg[i]), std::abs(du[i]), std::abs(dl[i])});
  uint8_t *pv = hs.piv + (size_t)(q - 1) * N;
  if (!band_lu(N, dl.data(), dg.data(), du.data(), du2.data(), pv)) return MDP_ERR_SINGULAR;
  double *F = hs.fact + (size_t)(q - 1) * N * FW;
  std::vector<uint8_t> isreal(N, 1);
  for (int i = 0; i < N; ++i) {
    if (std::abs(dg[i]) < kSingularTol * scale) return MDP_ERR_SINGULAR;
    const cd dinv = 1.0 / dg[i];
    const cd l = i < N - 1 ? dl[i] : cd(0.0);
    const cd u1 = i < N - 1 ? du[i] * dinv : cd(0.0);
    const cd u2 = i < N - 2 ? du2[i] * dinv : cd(0.0);
    // a factor entry whose imaginary part is below 2^-60 of its modulus is real to working
    // precision (the LU of an evanescent mode converges to real values away from the
    // Sommerfeld rows); such rows are stored exactly real and swept with real factors
    isreal[i] = tiny_imag(l) && tiny_imag(dinv) && tiny_imag(u1) && tiny_imag(u2);
    if (FW == 8) {
      F[i * 8 + 0] = l.real();    F[i * 8 + 1] = l.imag();
      F[i * 8 + 2] = dinv.real(); F[i * 8 + 3] = dinv.imag();
      F[i * 8 + 4] = u1.real();   F[i * 8 + 5] = u1.imag();
      F[i * 8 + 6] = u2.real();   F[i * 8 + 7] = u2.imag();
    } else {
      F[i * 4 + 0] = l.real(); F[i * 4 + 1] = dinv.real(); F[i * 4 + 2] = u1.real(); F[i * 4 + 3] = u2.real();
    }
  }
  // the longest run of real rows containing the middle row: [rlo, rhi)
  int rlo = N / 2, rhi = N / 2;
  if (FW == 8 && isreal[N / 2]) {
    rlo = N / 2; rhi = N / 2 + 1;
    while (rlo > 0 && isreal[rlo - 1]) --rlo;
    while (rhi < N && isreal[rhi]) ++rhi;
    for (int i = rlo; i < rhi; ++i)
      for (int w = 0; w < 4; ++w) F[i * 8 + 2 * w + 1] = 0.0;
  }
  if (FW == 4) { rlo = 0; rhi = N; }
  hs.seg[(size_t)(q - 1) * 5 + 0] = rlo;
  hs.seg[(size_t)(q - 1) * 5 + 1] = rhi;
  return build_fs_mode(hs, q);
}

static void prepare_tables(HostSub &hs) { hs.seg.assign((size_t)hs.d.Nq * 5, 0); }

// Factor every mode of every subdomain; modes are independent, so they are spread over the
// host's hardware threads (each writes its own table slices).
static mdp_status factor_all(std::vector<HostSub> &subs) {
  std::vector<std::pair<int, int>> tasks;
  for (int si = 0; si < (int)subs.size(); ++si) {
    prepare_tables(subs[si]);
    if (subs[si].d.leader != si) continue;   // a duplicate shares its leader's tables
    for (int q = 1; q <= subs[si].d.Nq; ++q) tasks.push_back({si, q});
  }
  const int nthr = (int)std::max(1u, std::min(std::thread::hardware_concurrency(), 64u));
  std::atomic<size_t> next(0);
  std::atomic<int> status(MDP_OK);
  auto worker = [&]() {
    for (;;) {
      const size_t t = next.fetch_add(1);
      if (t >= tasks.size() || status.load() != MDP_OK) return;
      const mdp_status st = factor_mode(subs[tasks[t].first], tasks[t].second);
      if (st != MDP_OK) status.store(st);
    }
  };
  std::vector<std::thread> pool;
  for (int i = 1; i < nthr; ++i) pool.emplace_back(worker);
  worker();
  for (auto &th : pool) th.join();
  for (int si = 0; si < (int)subs.size(); ++si)
    if (subs[si].d.leader != si) subs[si].seg = subs[subs[si].d.leader].seg;
  return (mdp_status)status.load();
}

// x = T_q^{-1} b (adjoint = 0) or T_q^{-H} b (adjoint = 1), complex interleaved host arrays,
// with the stored factors -- the same recurrences as the device kernels.
void host_mode_solve(const HostSub &hs, int q, int adjoint, const double *b, double *x) {
  const SubDesc &d = hs.d;
  const int N = d.Nt, FW = d.cplx ? 8 : 4;
  const double *F = hs.fact + (size_t)(q - 1) * N * FW;
  const uint8_t *pv = hs.piv + (size_t)(q - 1) * N;
  auto get = [&](int i, int w) -> cd {
    if (FW == 8) return cd(F[i * 8 + 2 * w], F[i * 8 + 2 * w + 1]);
    return cd(F[i * 4 + w], 0.0);
  };
  std::vector<cd> z(N);
  for (int i = 0; i < N; ++i) z[i] = cd(b[2 * i], b[2 * i + 1]);
  if (!adjoint) {
    for (int i = 0; i < N - 1; ++i) {
      if (pv[i]) std::swap(z[i], z[i + 1]);
      z[i + 1] -= get(i, 0) * z[i];
    }
    std::vector<cd> xs(N + 2, 0.0);
    for (int i = N - 1; i >= 0; --i) xs[i] = get(i, 1) * z[i] - get(i, 2) * xs[i + 1] - get(i, 3) * xs[i + 2];
    for (int i = 0; i < N; ++i) { x[2 * i] = xs[i].real(); x[2 * i + 1] = xs[i].imag(); }
  } else {
    // U^H z~ = b with z~_i = conj(d_i) z_i, then the transposed eliminations in reverse
    std::vector<cd> zt(N);
    for (int i = 0; i < N; ++i) {
      cd v = z[i];
      if (i >= 1) v -= std::conj(get(i - 1, 2)) * zt[i - 1];
      if (i >= 2) v -= std::conj(get(i - 2, 3)) * zt[i - 2];
      zt[i] = v;
    }
    for (int i = 0; i < N; ++i) z[i] = std::conj(get(i, 1)) * zt[i];
    for (int i = N - 2; i >= 0; --i) {
      z[i] -= std::conj(get(i, 0)) * z[i + 1];
      if (pv[i]) std::swap(z[i], z[i + 1]);
    }
    for (int i = 0; i < N; ++i) { x[2 * i] = z[i].real(); x[2 * i + 1] = z[i].imag(); }
  }
}

// ---------------------------------------------------------------- tables
static bool layout_tables(mdp_plan *p) {
  long long off = 0, poff = 0, out = 0;
  auto al = [](long long v) { return (v + 31) & ~31LL; };
  for (auto &hs : p->subs) {
    SubDesc &d = hs.d;
    if (d.leader != (int)(&hs - p->subs.data())) {   // a duplicate: the leader's tables
      const SubDesc &ld = p->subs[d.leader].d;
      d.fact_off = ld.fact_off; d.dT_off = ld.dT_off; d.sin_off = ld.sin_off; d.geo_off = ld.geo_off;
      d.seg_off = ld.seg_off; d.fs_off = ld.fs_off; d.piv_off = ld.piv_off; d.tcb_off = ld.tcb_off;
      d.out_off = out;  out += (long long)d.G * d.n_cols;
      continue;
    }
    const int FW = d.cplx ? 8 : 4;
    d.fact_off = off; off += al((long long)d.Nq * d.Nt * FW);
    d.dT_off = off;   off += al((long long)d.Nq * d.Nt * 6);
    d.sin_off = off;  off += al(4LL * d.Nx);
    d.geo_off = off;  off += al(4LL * d.G);
    d.seg_off = off;  off += al(5LL * d.Nq);
    d.fs_off = off;   off += al((long long)d.Nq * d.NYf * FSW);
    d.tcb_off = off;  off += d.tc_cols ? al(256LL * ((d.Nq + 15) / 16)) : 0;
    d.piv_off = poff; poff += al((long long)d.Nq * d.Nt);
    d.out_off = out;  out += (long long)d.G * d.n_cols;
  }
  const bool pinned = !(p->flags & MDP_PLAN_HOST_ONLY);
  if (!p->host_tables.alloc((size_t)off, pinned) || !p->host_piv.alloc((size_t)poff, pinned)) return false;
  for (auto &hs : p->subs) {
    const SubDesc &d = hs.d;
    hs.fact = p->host_tables.data() + d.fact_off;
    hs.dT = p->host_tables.data() + d.dT_off;
    hs.fs = p->host_tables.data() + d.fs_off;
    hs.piv = p->host_piv.data() + d.piv_off;
  }
  p->out_size = out;
  return true;
}

// fp16 bit pattern of the integer v, |v| <= 128 (exact)
static uint16_t f16_of_small_int(int v) {
  if (v == 0) return 0;
  const unsigned sgn = v < 0 ? 0x8000u : 0u;
  unsigned a = (unsigned)std::abs(v);
  int e = 0;
  while ((a >> (e + 1)) != 0) ++e;
  return (uint16_t)(sgn | ((unsigned)(e + 15) << 10) | ((a << (10 - e)) & 0x3FFu));
}

// The B operand of k_inv_cols_tc (the sine factors of the gamma-column sums) for every 16 modes:
// row n = 8 so + u holds digit u (u < 7; row 7 zero) of output so, where the outputs are, on a
// centred subdomain, sin(pi q m/Nx) at m = mlo-1, mlo for odd q, then the same for even q (zero
// at the other parity), else the columns mlo-1, mlo, mhi, mhi+1. A factor s becomes the integer
// W = round(s 2^50) through the bits of s + 6 (exact: |s| <= 1 keeps the sum in [4, 8)), written
// in 7 balanced base-256 digits (the bytes of W + 0x0080808080808080, each minus 128). Stored in
// the operand layout: 8 x 16-byte core matrices, K (the mode) fastest, 128 B between the two
// K halves and 256 B between groups of 8 rows.
// inner: the adjoint's ring columns mlo, mlo+1, mhi-1, mhi instead of the gamma columns
// mlo-1, mlo, mhi, mhi+1 (one column further in on either side)
static void fill_tc_block(const SubDesc &d, const double *S, uint16_t *blk, bool inner) {
  const int nch = (d.Nq + 15) / 16, N2 = 2 * d.Nx;
  int64_t magic, w;
  const double six = 6.0;
  std::memcpy(&magic, &six, 8);
  for (int c = 0; c < nch; ++c)
    for (int so = 0; so < 4; ++so)
      for (int kk = 0; kk < 16; ++kk) {
        const int q = c * 16 + 1 + kk;
        int m, par = -1;
        if (d.xsym) { m = ((so & 1) ? d.mlo : d.mlo - 1) + (inner ? 1 : 0); par = so < 2 ? 1 : 0; }
        else m = (so == 0 ? d.mlo - 1 : so == 1 ? d.mlo : so == 2 ? d.mhi : d.mhi + 1) + (inner ? (so < 2 ? 1 : -1) : 0);
        const double s = (q <= d.Nq && (par < 0 || (q & 1) == par)) ? S[(int)(((long long)q * m) % N2)] : 0.0;
        const double y = s + six;
        std::memcpy(&w, &y, 8);
        const uint64_t b = (uint64_t)(w - magic) + 0x0080808080808080ull;
        for (int u = 0; u < 8; ++u) {
          const int n = so * 8 + u;
          const int dig = u < 7 ? (int)((b >> (8 * (6 - u))) & 0xFF) - 128 : 0;
          blk[(size_t)c * 512 + (((n >> 3) * 256 + (kk >> 3) * 128 + (n & 7) * 16 + (kk & 7) * 2) >> 1)] =
              f16_of_small_int(dig);
        }
      }
}

static void fill_tables(mdp_plan *p) {
  for (auto &hs : p->subs) {
    const SubDesc &d = hs.d;
    if (d.leader != (int)(&hs - p->subs.data())) continue;
    double *S = &p->host_tables[d.sin_off];
    for (int j = 0; j < 2 * d.Nx; ++j) {
      S[j] = std::sin(M_PI * (double)j / (double)d.Nx);
      S[2 * d.Nx + j] = (2.0 / d.Nx) * S[j];
    }
    for (int i = 0; i < 5 * d.Nq; ++i) p->host_tables[d.seg_off + i] = hs.seg[i];
    if (d.tc_cols) {
      fill_tc_block(d, S, reinterpret_cast<uint16_t *>(&p->host_tables[d.tcb_off]), false);
      fill_tc_block(d, S, reinterpret_cast<uint16_t *>(&p->host_tables[d.tcb_off + 128LL * ((d.Nq + 15) / 16)]), true);
    }
    double *g = &p->host_tables[d.geo_off];
    for (int i = 0; i < d.G; ++i) {
      g[4 * i + 0] = hs.owner[i];
      g[4 * i + 1] = hs.s[i];
      g[4 * i + 2] = hs.rho[i];
      g[4 * i + 3] = hs.L[i];
    }
  }
}

static void schedule_pass(mdp_plan *p, bool grad, bool leaders_only, std::vector<Wave> &waves) {
  waves.clear();
  Wave cur;
  cur.ws_doubles = 0;
  const long long budget = p->ws_budget / 8;
  for (int si = 0; si < (int)p->subs.size(); ++si) {
    if (leaders_only && p->leader[si] != si) continue;
    const SubDesc &d = p->subs[si].d;
    for (int c0 = 0; c0 < d.n_cols; c0 += p->tile_cols) {
      Item it;
      std::memset(&it, 0, sizeof it);
      it.sub = si; it.col0 = c0; it.ncols = std::min(p->tile_cols, d.n_cols - c0);
      long long xi, r, gr, y, a, s, red, tot;
      item_workspace(d, it.ncols, grad, xi, r, gr, y, a, s, red, tot);
      if (!cur.items.empty() && cur.ws_doubles + tot > budget) {
        waves.push_back(cur);
        cur.items.clear();
        cur.ws_doubles = 0;
      }
      const long long base = cur.ws_doubles;
      it.xi_off = base + xi; it.r_off = base + r; it.gr_off = base + gr; it.y_off = base + y;
      it.a_off = base + a; it.s_off = base + s; it.red_off = base + red;
      it.io_off = d.out_off + (long long)c0 * d.G;
      cur.items.push_back(it);
      cur.ws_doubles += tot;
    }
  }
  if (!cur.items.empty()) waves.push_back(cur);
}

static void schedule(mdp_plan *p) {
  schedule_pass(p, false, false, p->sched[S_PROJ]);
  schedule_pass(p, true, false, p->sched[S_GRAD]);
  bool dups = false;
  for (int i = 0; i < (int)p->subs.size(); ++i) dups = dups || p->leader[i] != i;
  if (dups) schedule_pass(p, false, true, p->sched[S_BASIS]);
  else p->sched[S_BASIS].clear();
  long long mx = 0;
  for (auto &sc : p->sched)
    for (auto &w : sc) mx = std::max(mx, w.ws_doubles);
  p->ws_doubles = mx;
}

// Two subdomains pose the same auxiliary problem when they agree in every quantity the tables
// and the columns depend on: grid, step, wavenumber, AP type, modes, the index sets, and the
// gamma geometry relative to the grid (ownership, foot point, distance, side length) up to
// rounding of the placement.
static bool same_problem(const HostSub &a, const HostSub &b) {
  const SubDesc &x = a.d, &y = b.d;
  if (x.nx != y.nx || x.ny != y.ny || x.h != y.h || x.k != y.k || x.ap_bc != y.ap_bc || x.n_modes != y.n_modes ||
      x.mlo != y.mlo || x.mhi != y.mhi || x.nlo != y.nlo || x.nhi != y.nhi || x.G != y.G || x.nfirst != y.nfirst ||
      x.i0 != y.i0 || x.xsym != y.xsym)
    return false;
  const double tol = 1e-12 * x.h;
  for (int i = 0; i < x.G; ++i) {
    if (a.owner[i] != b.owner[i] || std::fabs(a.rho[i] - b.rho[i]) > tol || std::fabs(a.s[i] - b.s[i]) > 1e-12 ||
        std::fabs(a.L[i] - b.L[i]) > tol)
      return false;
  }
  return true;
}

static void find_leaders(mdp_plan *p) {
  const int n = (int)p->subs.size();
  p->leader.resize(n);
  for (int i = 0; i < n; ++i) {
    p->leader[i] = i;
    if (!(p->flags & MDP_PLAN_DEDUPE)) continue;
    for (int j = 0; j < i; ++j)
      if (p->leader[j] == j && same_problem(p->subs[i], p->subs[j])) { p->leader[i] = j; break; }
  }
  for (int i = 0; i < n; ++i) p->subs[i].d.leader = p->leader[i];
}

mdp_status build_host_plan(mdp_plan *p, const mdp_subdomain *subs, int n) {
  p->subs.resize(n);
  for (int i = 0; i < n; ++i) {
    mdp_status st = geometry(subs[i], p->subs[i], p->flags, p->fft_block_points);
    if (st != MDP_OK) return st;
  }
  find_leaders(p);
  p->fft_smem = 16;
  for (auto &hs : p->subs)
    if (hs.d.rows_fft) p->fft_smem = std::max(p->fft_smem, hs.d.fpb * 2 * hs.d.Nx * 16);
  if (!layout_tables(p)) return MDP_ERR_NOMEM;
  mdp_status st = factor_all(p->subs);
  if (st != MDP_OK) return st;
  fill_tables(p);
  schedule(p);
  return MDP_OK;
}

mdp_status set_k_fields(mdp_plan *p, const double *k) {
  for (int i = 0; i < (int)p->subs.size(); ++i) {
    if (!(k[i] > 0) || !std::isfinite(k[i])) return MDP_ERR_ARG;
    if (k[i] != k[p->leader[i]]) return MDP_ERR_ARG;   // deduplicated subdomains keep one k
  }
  for (int i = 0; i < (int)p->subs.size(); ++i) {
    HostSub &hs = p->subs[i];
    const double h2 = hs.d.h * hs.d.h, k2 = k[i] * k[i];
    hs.d.k = k[i];
    hs.d.c1 = 1.0 / h2 - 2.0 / (6.0 * h2) + k2 / 12.0;
    hs.d.c0 = -4.0 / h2 + 4.0 / (6.0 * h2) + 8.0 * k2 / 12.0;
    hs.d.dc1 = k[i] / 6.0;
    hs.d.dc0 = 8.0 * k[i] / 6.0;
  }
  return MDP_OK;
}

mdp_status refactor_host(mdp_plan *p, const double *k) {
  mdp_status st = set_k_fields(p, k);
  if (st != MDP_OK) return st;
  st = factor_all(p->subs);
  if (st != MDP_OK) return st;
  fill_tables(p);
  return MDP_OK;
}

}  // namespace mdp
