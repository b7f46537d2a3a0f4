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
#include <cstring>

namespace mdp {

using cd = std::complex<double>;

static const double kTieTol = 1e-9;       // side-ownership ties within 1e-9*h
static const double kSingularTol = 1e-13; // pivot below this x max|T| -> singular

const char *fam_name(int f) {
  static const char *names[NFAM] = {"k_extend", "k_residual", "k_fwd_rows", "k_tri", "k_inv_rows", "k_inv_cols",
                                    "k_adj_rows", "k_adj_tri", "k_adj_ring_rows", "k_adj_ring_cols", "k_adj_gamma",
                                    "k_inv_rec"};
  return (f >= 0 && f < NFAM) ? names[f] : "?";
}

void item_workspace(const SubDesc &d, int ncols, bool grad, long long &xi, long long &r, long long &gr,
                    long long &y, long long &a, long long &s, long long &red, long long &total) {
  auto al = [](long long v) { return (v + 31) & ~31LL; };  // 256-byte alignment (in doubles)
  long long off = 0;
  xi = off; off += al((long long)d.G * ncols * (grad ? 2 : 1));
  r = off;  off += al((long long)std::max(d.R, d.R2) * ncols * 2);
  gr = off; off += al(5LL * d.Nq * ncols * 2);  // 4 dense rows (+ the receiver row in the adjoint)
  y = off;  off += al((long long)d.Nq * (grad ? d.Nt : d.NYf) * ncols * 2);
  a = off;  off += grad ? al((long long)d.Nq * d.Nt * ncols * 2) : 0;
  s = off;  off += grad ? al((long long)d.R * ncols * 2) : 0;
  int rs[5];
  red_slots(d, ncols, rs);
  red = off; off += grad ? al(rs[4] + 1) : 0;
  total = off;
}

// ---------------------------------------------------------------- geometry
static mdp_status geometry(const mdp_subdomain &in, HostSub &hs) {
  SubDesc &d = hs.d;
  std::memset(&d, 0, sizeof d);
  if (in.nx < 9 || in.ny < 9 || !(in.h > 0) || !(in.k > 0) || in.n_modes < 1 ||
      (in.ap_bc != MDP_AP_DIRICHLET4 && in.ap_bc != MDP_AP_DIRX_SOMMY) || !(in.x1 > in.x0) ||
      !(in.y1 > in.y0) || !std::isfinite(in.k))
    return MDP_ERR_ARG;
  d.nx = in.nx; d.ny = in.ny; d.Nx = in.nx - 1; d.Nq = d.Nx - 1;
  d.h = in.h; d.k = in.k;
  d.x0 = in.x0; d.x1 = in.x1; d.y0 = in.y0; d.y1 = in.y1; d.ax0 = in.ax0; d.ay0 = in.ay0;
  d.ap_bc = in.ap_bc; d.cplx = in.ap_bc == MDP_AP_DIRX_SOMMY;
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
//   and the mirror image at n = 0.
// Factorisation: Gaussian elimination with partial pivoting on the band (row swaps create
// one extra super-diagonal), the textbook algorithm for banded LU.
static mdp_status factor_modes(HostSub &hs) {
  SubDesc &d = hs.d;
  const int N = d.Nt, FW = d.cplx ? 8 : 4;
  hs.fact.assign((size_t)d.Nq * N * FW, 0.0);
  hs.piv.assign((size_t)d.Nq * N, 0);
  hs.dT.assign((size_t)d.Nq * N * 6, 0.0);
  hs.seg.assign((size_t)d.Nq * 2, 0);
  const double h = d.h, h2 = h * h, k = d.k, k2 = k * k;
  std::vector<cd> dl(N), dg(N), du(N), du2(N);
  for (int q = 1; q <= d.Nq; ++q) {
    const double sq = std::sin(M_PI * q / (2.0 * d.Nx));
    const double lam = -4.0 * sq * sq;
    const double a = 1.0 / h2 + lam / (6.0 * h2) + k2 / 12.0;
    const double dd = -2.0 * a + lam / h2 + k2 + k2 * lam / 12.0;
    const double da = k / 6.0;
    const double ddd = -2.0 * da + 2.0 * k + 2.0 * k * lam / 12.0;
    const cd alpha((1.0 + k2 * h2 / 24.0 + lam / 24.0) / h2, 0.0);
    const cd beta(0.0, k * (1.0 + k2 * h2 / 8.0 + lam / 8.0) / h);
    const cd dalpha(k / 12.0, 0.0);
    const cd dbeta(0.0, (1.0 + 3.0 * k2 * h2 / 8.0 + lam / 8.0) / h);
    double *dT = &hs.dT[(size_t)(q - 1) * N * 6];
    for (int i = 0; i < N; ++i) {
      dl[i] = a; dg[i] = dd; du[i] = a; du2[i] = 0.0;
      cd tsub = da, tdg = ddd, tsup = da;
      if (d.cplx && i == 0) { dg[i] = alpha + 0.5 * beta; du[i] = -alpha + 0.5 * beta; tdg = dalpha + 0.5 * dbeta; tsup = -dalpha + 0.5 * dbeta; tsub = 0.0; }
      if (d.cplx && i == N - 1) { dg[i] = alpha + 0.5 * beta; tdg = dalpha + 0.5 * dbeta; tsub = -dalpha + 0.5 * dbeta; tsup = 0.0; }
      if (i == 0) tsub = 0.0;
      if (i == N - 1) tsup = 0.0;
      dT[i * 6 + 0] = tsub.real(); dT[i * 6 + 1] = tsub.imag();
      dT[i * 6 + 2] = tdg.real();  dT[i * 6 + 3] = tdg.imag();
      dT[i * 6 + 4] = tsup.real(); dT[i * 6 + 5] = tsup.imag();
    }
    // dl[i] is T[i+1][i]; the top Sommerfeld row's sub-diagonal entry is T[N-1][N-2]
    if (d.cplx) dl[N - 2] = -alpha + 0.5 * beta;
    double scale = 0.0;
    for (int i = 0; i < N; ++i) scale = std::max({scale, std::abs(dg[i]), std::abs(du[i]), std::abs(dl[i])});
    uint8_t *pv = &hs.piv[(size_t)(q - 1) * N];
    for (int i = 0; i < N - 1; ++i) {
      if (std::abs(dg[i]) >= std::abs(dl[i])) {
        if (dg[i] == 0.0) return MDP_ERR_SINGULAR;
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
    double *F = &hs.fact[(size_t)(q - 1) * N * FW];
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
      auto tiny = [](cd v) { return std::fabs(v.imag()) <= 0x1p-60 * std::abs(v); };
      isreal[i] = tiny(l) && tiny(dinv) && tiny(u1) && tiny(u2);
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
    hs.seg[(size_t)(q - 1) * 2 + 0] = rlo;
    hs.seg[(size_t)(q - 1) * 2 + 1] = rhi;
  }
  return MDP_OK;
}

// x = T_q^{-1} b (adjoint = 0) or T_q^{-H} b (adjoint = 1), complex interleaved host arrays,
// with the stored factors -- the same recurrences as the device kernels.
void host_mode_solve(const HostSub &hs, int q, int adjoint, const double *b, double *x) {
  const SubDesc &d = hs.d;
  const int N = d.Nt, FW = d.cplx ? 8 : 4;
  const double *F = &hs.fact[(size_t)(q - 1) * N * FW];
  const uint8_t *pv = &hs.piv[(size_t)(q - 1) * N];
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
static void layout_tables(mdp_plan *p) {
  long long off = 0, poff = 0, out = 0;
  auto al = [](long long v) { return (v + 31) & ~31LL; };
  for (auto &hs : p->subs) {
    SubDesc &d = hs.d;
    const int FW = d.cplx ? 8 : 4;
    d.fact_off = off; off += al((long long)d.Nq * d.Nt * FW);
    d.dT_off = off;   off += al((long long)d.Nq * d.Nt * 6);
    d.sin_off = off;  off += al(4LL * d.Nx);
    d.geo_off = off;  off += al(4LL * d.G);
    d.seg_off = off;  off += al(2LL * d.Nq);
    d.piv_off = poff; poff += al((long long)d.Nq * d.Nt);
    d.out_off = out;  out += (long long)d.G * d.n_cols;
  }
  p->host_tables.assign(off, 0.0);
  p->host_piv.assign(poff, 0);
  p->out_size = out;
}

static void fill_tables(mdp_plan *p) {
  for (auto &hs : p->subs) {
    const SubDesc &d = hs.d;
    std::copy(hs.fact.begin(), hs.fact.end(), p->host_tables.begin() + d.fact_off);
    std::copy(hs.dT.begin(), hs.dT.end(), p->host_tables.begin() + d.dT_off);
    std::copy(hs.piv.begin(), hs.piv.end(), p->host_piv.begin() + d.piv_off);
    double *S = &p->host_tables[d.sin_off];
    for (int j = 0; j < 2 * d.Nx; ++j) {
      S[j] = std::sin(M_PI * (double)j / (double)d.Nx);
      S[2 * d.Nx + j] = (2.0 / d.Nx) * S[j];
    }
    for (int i = 0; i < 2 * d.Nq; ++i) p->host_tables[d.seg_off + i] = hs.seg[i];
    double *g = &p->host_tables[d.geo_off];
    for (int i = 0; i < d.G; ++i) {
      g[4 * i + 0] = hs.owner[i];
      g[4 * i + 1] = hs.s[i];
      g[4 * i + 2] = hs.rho[i];
      g[4 * i + 3] = hs.L[i];
    }
  }
}

static void schedule_pass(mdp_plan *p, bool grad, std::vector<Wave> &waves) {
  waves.clear();
  Wave cur;
  cur.ws_doubles = 0;
  const long long budget = p->ws_budget / 8;
  for (int si = 0; si < (int)p->subs.size(); ++si) {
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
  schedule_pass(p, false, p->waves);
  schedule_pass(p, true, p->gwaves);
  long long mx = 0;
  for (auto &w : p->waves) mx = std::max(mx, w.ws_doubles);
  for (auto &w : p->gwaves) mx = std::max(mx, w.ws_doubles);
  p->ws_doubles = mx;
}

mdp_status build_host_plan(mdp_plan *p, const mdp_subdomain *subs, int n) {
  p->subs.resize(n);
  for (int i = 0; i < n; ++i) {
    mdp_status st = geometry(subs[i], p->subs[i]);
    if (st != MDP_OK) return st;
    st = factor_modes(p->subs[i]);
    if (st != MDP_OK) return st;
  }
  layout_tables(p);
  fill_tables(p);
  schedule(p);
  return MDP_OK;
}

mdp_status refactor_host(mdp_plan *p, const double *k) {
  for (int i = 0; i < (int)p->subs.size(); ++i) {
    if (!(k[i] > 0) || !std::isfinite(k[i])) return MDP_ERR_ARG;
  }
  for (int i = 0; i < (int)p->subs.size(); ++i) {
    HostSub &hs = p->subs[i];
    SubDesc keep = hs.d;
    const double h2 = keep.h * keep.h, k2 = k[i] * k[i];
    hs.d.k = k[i];
    hs.d.c1 = 1.0 / h2 - 2.0 / (6.0 * h2) + k2 / 12.0;
    hs.d.c0 = -4.0 / h2 + 4.0 / (6.0 * h2) + 8.0 * k2 / 12.0;
    hs.d.dc1 = k[i] / 6.0;
    hs.d.dc0 = 8.0 * k[i] / 6.0;
    mdp_status st = factor_modes(hs);
    if (st != MDP_OK) return st;
  }
  fill_tables(p);
  return MDP_OK;
}

}  // namespace mdp
