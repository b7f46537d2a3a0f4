// CUDA kernels (sm_103a, FP64) of the batched projection columns:
//   k_extend    basis + equation-based extension on gamma       (Sections 3.2.3-3.2.4)
//   k_residual  r = L^(h) w restricted to M+ (the 2-node ring)   (Eqs. FD_scheme, Potential_def)
//   k_fwd_rows  sine transform along x of the 4 dense ring rows  (Section 3.2.1 / 3.6: "sine-FFT")
//   k_tri       per-mode pivoted tridiagonal solve along y; the sine transform of the ring's
//               middle rows (4 nonzeros per row) is fused into its forward sweep
//   k_inv_rows  inverse sine transform onto the 4 full gamma rows, column output
//   k_inv_cols  inverse sine transform onto the 4 gamma columns of the middle rows
// Q column = -Tr G^(h) r, P_gamma column = xi - Tr G^(h) r (Eqs. def_Pgamma, Q_construction).
//
// Every kernel takes a Batch: blocks are numbered across all work items of the launch and
// each block finds its item by binary search over a prefix array. Within an item, the block
// is (32 columns) x (BY tasks): a warp shares one task (one mode, one row ...), so factor and
// sine-table loads are warp-uniform broadcasts and column data is read coalesced.
#include "kernels_common.cuh"

#include <algorithm>
#include <cstring>

namespace mdp {

// ---------------------------------------------------------------- k_extend
// One thread per gamma node: the Chebyshev recurrences for T_j, T_j'', T_j'''' (with T', T'''
// as intermediates) run once over j and serve every column of the owner side in the item.
// Writes xi[g][c - col0] (real) for those columns; with grad also d xi / dk after G*ncols.
__global__ void __launch_bounds__(128) k_extend(Batch bt, const SubDesc *subs, const double *tab, double *ws, int grad) {
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_EXT);
  const SubDesc &d = subs[it.sub];
  const int g = local * 128 + threadIdx.x;
  if (g >= d.G) return;
  const double *geo = tab + d.geo_off + 4 * g;
  const int side = (int)geo[0];
  const double s = geo[1], rho = geo[2], L = geo[3];
  const int M = d.n_modes;
  const int baseD = (side - 1) * M, baseN = 4 * M + (side - 1) * M;
  const int c0 = it.col0, c1 = it.col0 + it.ncols;
  // j range needed: any j with baseD + j or baseN + j inside [c0, c1)
  int jmax = 0;
  if (c1 > baseD) jmax = max(jmax, min(M, c1 - baseD));
  if (c1 > baseN) jmax = max(jmax, min(M, c1 - baseN));
  double *xi = ws + it.xi_off;
  const double k = d.k, k2 = k * k, k4 = k2 * k2;
  const double sc2 = (2.0 / L) * (2.0 / L), sc4 = sc2 * sc2;
  const double a2 = 0.5 * rho * rho, a4 = a2 * a2 / 6.0, a3 = a2 * rho / 3.0;
  double t0 = 1.0, t1 = 0.0, t2 = 0.0, t3 = 0.0, t4 = 0.0;
  double p0 = 0.0, p1 = 0.0, p2 = 0.0, p3 = 0.0, p4 = 0.0;
  const double s2 = 2.0 * s;
  for (int j = 0; j < jmax; ++j) {
    const double psi = t0, psi2 = t2 * sc2, psi4 = t4 * sc4;
    const double tt = fma(-k2, psi, -psi2);                // -psi'' - k^2 psi
    const int cD = baseD + j, cN = baseN + j;
    if (cD >= c0 && cD < c1) {
      const double v4 = fma(k4, psi, fma(2.0 * k2, psi2, psi4));
      xi[(long long)g * it.ncols + (cD - c0)] = fma(a4, v4, fma(a2, tt, psi));
      if (grad) xi[(long long)d.G * it.ncols + (long long)g * it.ncols + (cD - c0)] =
          fma(a2, -2.0 * k * psi, a4 * (4.0 * k * psi2 + 4.0 * k * k2 * psi));
    }
    if (cN >= c0 && cN < c1) {
      xi[(long long)g * it.ncols + (cN - c0)] = fma(a3, tt, rho * psi);
      if (grad) xi[(long long)d.G * it.ncols + (long long)g * it.ncols + (cN - c0)] = a3 * (-2.0 * k * psi);
    }
    double n0, n1, n2, n3, n4;
    if (j == 0) { n0 = s; n1 = 1.0; n2 = 0.0; n3 = 0.0; n4 = 0.0; }
    else {
      n0 = fma(s2, t0, -p0);
      n1 = fma(s2, t1, fma(2.0, t0, -p1));
      n2 = fma(s2, t2, fma(4.0, t1, -p2));
      n3 = fma(s2, t3, fma(6.0, t2, -p3));
      n4 = fma(s2, t4, fma(8.0, t3, -p4));
    }
    p0 = t0; p1 = t1; p2 = t2; p3 = t3; p4 = t4;
    t0 = n0; t1 = n1; t2 = n2; t3 = n3; t4 = n4;
  }
}

// ---------------------------------------------------------------- k_residual
// r(ring node) = sum over the 3x3 stencil of the gamma neighbours (w = xi on gamma, 0 elsewhere).
// With GRAD also s = (dL/dk w + L dw/dk)(ring node) (dw/dk: the extension's k-dependence, basis).
template <bool CIN, bool GRAD>
__device__ __forceinline__ cplx ring_stencil(const SubDesc &d, const Item &it, const double *ws, const double *tab,
                                             const double2 *xi_user, int b, int n, int m, cplx *s_out) {
  const int side = col_side(d, it.col0 + b);
  const double *dxi = ws + it.xi_off + (long long)d.G * it.ncols;
  cplx acc = cmk(0.0, 0.0), sacc = cmk(0.0, 0.0);
#pragma unroll
  for (int dn = -1; dn <= 1; ++dn) {
#pragma unroll
    for (int dm = -1; dm <= 1; ++dm) {
      const int g = gamma_index(d, n + dn, m + dm);
      if (g < 0) continue;
      const int nb = (dn != 0) + (dm != 0);
      const double c = nb == 0 ? d.c0 : nb == 1 ? d.c1 : d.c2;
      const cplx v = density<CIN>(d, it, ws, tab, xi_user, b, g);
      acc = caxpy(c, v, acc);
      if (GRAD) {
        const double dc = nb == 0 ? d.dc0 : nb == 1 ? d.dc1 : 0.0;
        sacc = caxpy(dc, v, sacc);
        if (!CIN && (int)tab[d.geo_off + 4 * g] == side) sacc.re = fma(c, dxi[(long long)g * it.ncols + b], sacc.re);
      }
    }
  }
  if (GRAD) *s_out = sacc;
  return acc;
}

// One thread per (ring unit, column). Plain layout: a unit is one ring node, r[ri][b]. Centred
// subdomains (xsym): a unit is the node pair (m, Nx - m) of a ring row, stored as
// (r(m) + r(Nx-m), r(m) - r(Nx-m)) -- 4 Ph dense-row units and 2 per middle row -- so that
// the sine transforms need one product per pair. The gradient's s is stored plain [ri][b].
template <bool CIN, bool GRAD>
__global__ void __launch_bounds__(256) k_residual(Batch bt, const SubDesc *subs, const double *tab, double *ws,
                                                  const double2 *xi_user) {
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_RES);
  const SubDesc &d = subs[it.sub];
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int u = (local / cb) * 8 + threadIdx.y;
  const int units = d.xsym ? 4 * d.Ph + 2 * (d.Py - 4) : d.R;
  if (!GRAD && u == 0 && b < it.ncols && d.tc_cols) reinterpret_cast<int *>(ws + it.red_off)[b] = 0;  // for k_tri
  if (b >= it.ncols || u >= units) return;
  double *r = ws + it.r_off;
  double *sb = ws + it.s_off;
  const long long nc = it.ncols;
  if (!d.xsym) {
    int n, m;
    ring_node(d, u, n, m);
    cplx sv;
    const cplx v = ring_stencil<CIN, GRAD>(d, it, ws, tab, xi_user, b, n, m, &sv);
    if (CIN) st2(r + 2 * (u * nc + b), v); else r[u * nc + b] = v.re;
    if (GRAD) st2(sb + 2 * (u * nc + b), sv);
    return;
  }
  int n, m1, slot;
  if (u < 4 * d.Ph) {
    const int rr = u / d.Ph, k = u % d.Ph;
    n = rr == 0 ? d.nlo : rr == 1 ? d.nlo + 1 : rr == 2 ? d.nhi - 1 : d.nhi;
    m1 = d.mlo + k;
    slot = rr * 2 * d.Ph + 2 * k;
  } else {
    const int t = (u - 4 * d.Ph) >> 1, pr = (u - 4 * d.Ph) & 1;
    n = d.nlo + 2 + t;
    m1 = d.mlo + pr;
    slot = 8 * d.Ph + 4 * t + 2 * pr;
  }
  const int m2 = d.Nx - m1;
  cplx s1, s2 = cmk(0.0, 0.0);
  const cplx v1 = ring_stencil<CIN, GRAD>(d, it, ws, tab, xi_user, b, n, m1, &s1);
  const cplx v2 = m2 != m1 ? ring_stencil<CIN, GRAD>(d, it, ws, tab, xi_user, b, n, m2, &s2) : cmk(0.0, 0.0);
  const cplx vp = cadd(v1, v2), vm = csub(v1, v2);
  if (CIN) { st2(r + 2 * (slot * nc + b), vp); st2(r + 2 * ((slot + 1) * nc + b), vm); }
  else { r[slot * nc + b] = vp.re; r[(slot + 1) * nc + b] = vm.re; }
  if (GRAD) {
    st2(sb + 2 * ((long long)ring_index(d, n, m1) * nc + b), s1);
    if (m2 != m1) st2(sb + 2 * ((long long)ring_index(d, n, m2) * nc + b), s2);
  }
}

// ---------------------------------------------------------------- k_fwd_rows
// ghat(q, row) = sum_m sin(pi q m / Nx) r(m, row) for the 4 dense ring rows.
//
// FFT form (Nx a power of 2): a DST-I by one complex FFT of length Nx (dst1_post). Real ring
// data (basis columns) pack two rows of the same column per transform, x = r_a + i r_b (rows
// nlo, nlo+1 and nhi-1, nhi): the transform is linear with real coefficients, so ghat_a = Re F
// and ghat_b = Im F, and a column's result does not depend on its neighbours. One block: one
// ring row (or row pair) and fpb columns.
//
// Direct form: a thread handles the mode pair (q, Nx - q): sin(pi (Nx-q) m/Nx) =
// (-1)^(m+1) sin(pi q m/Nx), so the odd-m and even-m partial sums give both modes.
template <bool CIN>
__device__ __forceinline__ void fwd_rows_fft(const Item &it, const SubDesc &d, const double *tab, double *ws,
                                             int local, double2 *sm) {
  __shared__ double2 tot[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int rr = local & 3, cblk = local >> 2;
  if (!CIN && (rr & 1)) return;                        // real data: rows rr, rr + 1 in one block
  const int b0 = cblk * d.fpb, nf = min(d.fpb, it.ncols - b0);
  const int N = d.Nx, H = N / 2;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  const double *sn = tab + d.sin_off;
  const double *r = ws + it.r_off;
  const long long nc = it.ncols;
  const int P = d.Px, Mr = 4 * (d.Py - 4);
  auto rv = [&](long long slot, int b) -> cplx { return CIN ? ld2(r + 2 * (slot * nc + b)) : cmk(r[slot * nc + b], 0.0); };
  // (x_j + x_{N-j}, x_j - x_{N-j}) of ring row `row`, column b, j = 1 .. N/2: x-centred
  // subdomains store exactly these pairs for j in [mlo, N/2] (at j = N/2 both slots hold r)
  auto pm = [&](int row, int j, int b, cplx &p, cplx &m) {
    if (d.xsym) {
      if (j < d.mlo) { p = m = cmk(0.0, 0.0); return; }
      const long long slot = (long long)row * 2 * d.Ph + 2 * (j - d.mlo);
      p = rv(slot, b);
      m = 2 * j == N ? cmk(0.0, 0.0) : rv(slot + 1, b);
      if (2 * j == N) p = cmk(2.0 * p.re, 2.0 * p.im);
      return;
    }
    const int rb = row == 0 ? 0 : row == 1 ? P : row == 2 ? 2 * P + Mr : 3 * P + Mr;
    const cplx xa = (j >= d.mlo && j <= d.mhi) ? rv(rb + (j - d.mlo), b) : cmk(0.0, 0.0);
    const cplx xb = (N - j >= d.mlo && N - j <= d.mhi) ? rv(rb + (N - j - d.mlo), b) : cmk(0.0, 0.0);
    p = cadd(xa, xb);
    m = 2 * j == N ? cmk(0.0, 0.0) : csub(xa, xb);
  };
  // the twisted sequence y, bit-reversed, for the pairs (j, N - j)
  for (int idx = tid; idx < d.fpb * (H + 1); idx += nt) {
    const int f = idx / (H + 1), j = idx - f * (H + 1);
    double2 *S = sm + (long long)f * N;
    if (j == 0) { S[0] = make_double2(0.0, 0.0); continue; }
    cplx p = cmk(0.0, 0.0), m = cmk(0.0, 0.0);
    if (f < nf) {
      if (CIN) {
        pm(rr, j, b0 + f, p, m);
      } else {   // rows rr (real part) and rr + 1 (imaginary part)
        cplx p1, m1;
        pm(rr, j, b0 + f, p, m);
        pm(rr + 1, j, b0 + f, p1, m1);
        p = cmk(p.re, p1.re);
        m = cmk(m.re, m1.re);
      }
    }
    if (2 * j == N) { S[brev_lg(j, lg)] = make_double2(p.re, p.im); continue; }   // y_{N/2} = 2 x_{N/2}
    const double sj = sn[j];
    S[brev_lg(j, lg)] = make_double2(fma(sj, p.re, 0.5 * m.re), fma(sj, p.im, 0.5 * m.im));
    S[brev_lg(N - j, lg)] = make_double2(fma(sj, p.re, -0.5 * m.re), fma(sj, p.im, -0.5 * m.im));
  }
  __syncthreads();
  fft_r2_stages(sm, d.fpb, N, lg, sn);
  double2 *F = sm + (long long)d.fpb * N;
  dst1_post(sm, F, d.fpb, N, tot);
  double *gr = ws + it.gr_off;
  for (int idx = tid; idx < nf * d.Nq; idx += nt) {
    const int f = idx % nf, q = idx / nf + 1;
    const double2 V = F[(long long)f * N + q];
    const long long o = ((long long)rr * d.Nq + (q - 1)) * nc + b0 + f;
    if (CIN) {
      st2(gr + 2 * o, cmk(V.x, V.y));
    } else {
      gr[o] = V.x;
      gr[o + (long long)d.Nq * nc] = V.y;       // row rr + 1
    }
  }
}

template <bool CIN>
__global__ void __launch_bounds__(256) k_fwd_rows(Batch bt, const SubDesc *subs, const double *tab, double *ws) {
  extern __shared__ double2 fft_sm[];
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_FROWS);
  const SubDesc &d = subs[it.sub];
  if (d.rows_fft) { fwd_rows_fft<CIN>(it, d, tab, ws, local, fft_sm); return; }
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int q = (local / cb) * 8 + threadIdx.y + 1;
  if (b >= it.ncols || q > d.Nx / 2) return;
  const double *S = tab + d.sin_off;
  const int N2 = 2 * d.Nx, P = d.Px, Mr = 4 * (d.Py - 4);
  const double *r = ws + it.r_off;
  double *gr = ws + it.gr_off;
  const int q2 = d.Nx - q;
  const int par = (q & 1) ? 0 : 1;  // xsym: odd modes use r(m) + r(Nx-m), even modes the difference
  for (int rr = 0; rr < 4; ++rr) {
    const int rb = rr == 0 ? 0 : rr == 1 ? P : rr == 2 ? 2 * P + Mr : 3 * P + Mr;
    cplx ao = cmk(0.0, 0.0), ae = cmk(0.0, 0.0);
    int j = (int)(((long long)q * d.mlo) % N2);
    const int cnt = d.xsym ? d.Ph : P;
    for (int mm = 0; mm < cnt; ++mm) {
      const int m = d.mlo + mm;
      const double sv = S[j];
      const long long slot = d.xsym ? (long long)rr * 2 * d.Ph + 2 * mm + par : rb + mm;
      cplx v;
      if (CIN) v = ld2(r + 2 * (slot * it.ncols + b));
      else v = cmk(r[slot * it.ncols + b], 0.0);
      if (m & 1) ao = caxpy(sv, v, ao); else ae = caxpy(sv, v, ae);
      j += q;
      if (j >= N2) j -= N2;
    }
    const long long o1 = ((long long)rr * d.Nq + (q - 1)) * it.ncols + b;
    const long long o2 = ((long long)rr * d.Nq + (q2 - 1)) * it.ncols + b;
    if (CIN) {
      st2(gr + 2 * o1, cadd(ao, ae));
      if (q2 != q) st2(gr + 2 * o2, csub(ao, ae));
    } else {
      gr[o1] = ao.re + ae.re;
      if (q2 != q) gr[o2] = ao.re - ae.re;
    }
  }
}

// ---------------------------------------------------------------- k_tri
// The gradient pass's forward recompute: per (mode q, column b) the full pivoted LU sweep over
// every row -- forward elimination with the stored row swaps from matrix row i0 (rows below carry
// zero right-hand side) to the top, then back substitution down to row 0, every row stored as
// y[q-1][i][b] (complex). RHS at grid row n: the dense ring rows read ghat; the middle ring rows
// have 4 nonzeros (columns mlo, mlo+1, mhi-1, mhi), so their sine transform is 4 products here.
// CF: complex factors (Sommerfeld AP). CIN: complex ring data. Factor rows [rlo, rhi) of a
// complex AP are real to working precision (set by the plan): there the sweeps use real factors,
// and the forward sweep stays in real arithmetic while the data are still real (real densities,
// no complex factor row met yet). The forward sweep stores y~_i = y_i / d_i (the pivot's
// reciprocal is in the staged factor row), so the back substitution is x_i = y~_i - u1 x_{i+1}
// - u2 x_{i+2} with no product by 1/d; while the data are real, y~ is stored packed as in the
// projection sweep. Operands are staged 2 rows ahead: the factor row, the 4-byte word holding
// the row's swap flag, and the lane's ring values (forward) or stored y~ (back).
template <bool CIN>
__host__ __device__ constexpr int full_stage_bytes() { return 80 + 4 * 32 * (CIN ? 16 : 8); }

template <bool CF, bool CIN>
__device__ __forceinline__ void tri_full_body(const Item &it, const SubDesc &d, const double *tab, const uint8_t *pivtab,
                                              double *ws, int b, int q, char *sw, int lane, int nact, unsigned mask) {
  constexpr int FW = CF ? 8 : 4, VS = CIN ? 16 : 8, SB = full_stage_bytes<CIN>(), RING = 80;
  constexpr int TRI_D = 2;   // stages per warp
  // descriptor fields in registers (the copies' memory clobbers would otherwise reload them)
  const int i0 = d.i0, nfirst = d.nfirst, nlo = d.nlo, nhi = d.nhi, Nq = d.Nq, Ph = d.Ph, Nt = d.Nt;
  const bool xsym = d.xsym;
  const int N2 = 2 * d.Nx;
  const double *S = tab + d.sin_off;
  const double sm0 = S[(q * d.mlo) % N2], sm1 = S[(q * (d.mlo + 1)) % N2];
  const double sm2 = S[(q * (d.mhi - 1)) % N2], sm3 = S[(q * d.mhi) % N2];
  const int par = (q & 1) ? 0 : 1;
  const double *F = tab + d.fact_off + (long long)(q - 1) * Nt * FW;
  const uint8_t *pv = pivtab + d.piv_off + (long long)(q - 1) * Nt;
  const double *r = ws + it.r_off;
  const double *gr = ws + it.gr_off;
  double *y = ws + it.y_off;
  const int P = d.Px, nc = it.ncols;
  const long long ybase = (long long)(q - 1) * Nt * nc + b;
  int rlo = 0, rhi = Nt;  // real factor rows
  if (CF) {
    const double *sg = tab + d.seg_off + 5 * (q - 1);
    rlo = (int)sg[0];
    rhi = (int)sg[1];
  }
  auto ystore = [&](int i, cplx v) { st2(y + 2 * (ybase + (long long)i * nc), v); };
  // a real y~ of the warp's 32 columns packed into the first half of their complex slots of row
  // i (the back substitution stores x over them after every lane's copy of row i has landed)
  auto ystore_re = [&](int i, double v) { y[2 * (ybase + (long long)i * nc) - lane] = v; };
  int ipack = i0;   // rows i0 .. ipack-1 hold packed real y~
  auto dense = [&](int n) -> int {
    return n == nlo ? 0 : n == nlo + 1 ? 1 : n == nhi - 1 ? 2 : n == nhi ? 3 : -1;
  };
  auto stage = [&](int i) -> char * { return sw + (i & (TRI_D - 1)) * SB; };
  // the factor row and the word holding the row's swap flag (the flag table is 4-byte aligned
  // and padded to a multiple of 32 bytes, so the word never leaves it)
  auto fetch_row = [&](char *st, int i) {
    const double *src = F + (long long)i * FW;
    if (nact >= FW / 2) {
      if (lane < FW / 2) cp_async16(st + 16 * lane, src + 2 * lane);
    } else {
      for (int c = lane; c < FW / 2; c += nact) cp_async16(st + 16 * c, src + 2 * c);
    }
    if (lane == 0) {
      const uintptr_t a = reinterpret_cast<uintptr_t>(pv + i);
      cp_async4(st + 64, reinterpret_cast<const void *>(a & ~(uintptr_t)3));
    }
  };
  auto flag = [&](const char *st, int i) -> bool {
    const unsigned w = *reinterpret_cast<const unsigned *>(st + 64);
    return ((w >> (8 * (reinterpret_cast<uintptr_t>(pv + i) & 3))) & 0xffu) != 0;
  };
  // ---- forward staging: factor row, flag word, ring values of grid row n = i + 1 + nfirst
  auto fetch_fwd = [&](int i) {
    char *st = stage(i);
    fetch_row(st, i);
    const int n = i + 1 + nfirst;
    if (n >= nlo && n <= nhi) {
      char *rb = st + RING + VS * lane;
      auto cpv = [&](int slot, const double *base, long long o) {
        if (CIN) cp_async16(rb + slot * 32 * VS, base + 2 * o); else cp_async8(rb + slot * 32 * VS, base + o);
      };
      const int rr = dense(n);
      if (rr >= 0) {
        cpv(0, gr, ((long long)rr * Nq + (q - 1)) * nc + b);
      } else if (xsym) {
        const long long base = 8LL * Ph + 4 * (n - nlo - 2) + par;
        cpv(0, r, base * nc + b);
        cpv(1, r, (base + 2) * nc + b);
      } else {
        const long long ri = 2 * P + 4 * (n - nlo - 2);
        for (int s_ = 0; s_ < 4; ++s_) cpv(s_, r, (ri + s_) * nc + b);
      }
    }
    cp_async_commit();
  };
  auto sv = [&](const char *st, int slot) -> cplx {
    const double *p = reinterpret_cast<const double *>(st + RING + VS * lane + slot * 32 * VS);
    return CIN ? ld2(p) : cmk(p[0], 0.0);
  };
  // right-hand side of grid row n from the staged ring values (real data: the real part only,
  // as in the projection sweep)
  auto rhs = [&](const char *st, int n) -> cplx {
    if (n < nlo || n > nhi) return cmk(0.0, 0.0);
    if (dense(n) >= 0) return sv(st, 0);
    if (!CIN) {
      if (xsym) return cmk(fma(sm1, sv(st, 1).re, sm0 * sv(st, 0).re), 0.0);
      double v = sm0 * sv(st, 0).re;
      v = fma(sm1, sv(st, 1).re, v); v = fma(sm2, sv(st, 2).re, v); v = fma(sm3, sv(st, 3).re, v);
      return cmk(v, 0.0);
    }
    if (xsym) {
      const cplx v0 = sv(st, 0);
      return caxpy(sm1, sv(st, 1), cmk(sm0 * v0.re, sm0 * v0.im));
    }
    cplx v = cmk(0.0, 0.0);
    v = caxpy(sm0, sv(st, 0), v); v = caxpy(sm1, sv(st, 1), v); v = caxpy(sm2, sv(st, 2), v); v = caxpy(sm3, sv(st, 3), v);
    return v;
  };
  const int iend = Nt - 1;
  auto begin = [&](int i) -> const char * {
    cp_async_wait<TRI_D - 1>();
    __syncwarp(mask);
    return stage(i);
  };
  auto end_fwd = [&](int i) {
    __syncwarp(mask);
    if (i + TRI_D < iend) fetch_fwd(i + TRI_D); else cp_async_commit();
  };
  for (int j = 0; j < TRI_D; ++j) {
    if (i0 + j < iend) fetch_fwd(i0 + j); else cp_async_commit();
  }
  // ---- forward sweep: cur holds the eliminated value of row i
  cplx cur = cmk(0.0, 0.0);
  int i = i0;
  auto fwd_complex = [&](int i) {
    const char *st = begin(i);
    const double *row = reinterpret_cast<const double *>(st);
    const cplx g = rhs(st, i + 1 + nfirst);
    const cplx l = ld2(row);
    cplx yv;
    if (flag(st, i)) { yv = g; cur = cfms(cur, l, g); } else { yv = cur; cur = cfms(g, l, cur); }
    ystore(i, cmul(ld2(row + 2), yv));
    end_fwd(i);
  };
  if (CF) {  // complex factor rows below the real run
    const int e = min(max(rlo, i0), iend);
    for (; i < e; ++i) fwd_complex(i);
  }
  {
    const int e = min(max(rhi, i), iend);
    const bool realdata = !CIN && !(CF && i > i0);  // nothing complex has entered cur yet
    if (realdata) {
      for (; i < e; ++i) {
        const char *st = begin(i);
        const double g = rhs(st, i + 1 + nfirst).re;
        const double l = reinterpret_cast<const double *>(st)[0], dinv = reinterpret_cast<const double *>(st)[CF ? 2 : 1];
        double yv;
        if (flag(st, i)) { yv = g; cur.re = fma(-l, g, cur.re); } else { yv = cur.re; cur.re = fma(-l, cur.re, g); }
        ystore_re(i, dinv * yv);
        end_fwd(i);
      }
      ipack = i;
    } else {
      for (; i < e; ++i) {
        const char *st = begin(i);
        const cplx g = rhs(st, i + 1 + nfirst);
        const double l = reinterpret_cast<const double *>(st)[0], dinv = reinterpret_cast<const double *>(st)[CF ? 2 : 1];
        cplx yv;
        if (flag(st, i)) { yv = g; cur = caxpy(-l, g, cur); } else { yv = cur; cur = caxpy(-l, cur, g); }
        ystore(i, cmk(dinv * yv.re, dinv * yv.im));
        end_fwd(i);
      }
    }
  }
  if (CF)  // complex factor rows above the real run
    for (; i < iend; ++i) fwd_complex(i);
  {  // the top row's pivot is not staged by the forward sweep
    const double *rt = F + (long long)iend * FW;
    ystore(iend, CF ? cmul(ld2(rt + 2), cur) : cmk(rt[1] * cur.re, rt[1] * cur.im));
  }
  // the stored rows are read back below by this thread's asynchronous copies: order them after
  // its stores
  __threadfence_block();
  // ---- back substitution, every row stored (rows below i0 have zero eliminated right-hand side)
  auto fetch_back = [&](int i) {
    char *st = stage(i);
    fetch_row(st, i);
    if (i >= ipack) cp_async16(st + RING + 16 * lane, y + 2 * (ybase + (long long)i * nc));
    else if (i >= i0) cp_async8(st + RING + 16 * lane, y + 2 * (ybase + (long long)i * nc) - lane);
    cp_async_commit();
  };
  auto end_back = [&](int i) {
    __syncwarp(mask);
    if (i - TRI_D >= 0) fetch_back(i - TRI_D); else cp_async_commit();
  };
  for (int j = 0; j < TRI_D; ++j) {
    if (iend - j >= 0) fetch_back(iend - j); else cp_async_commit();
  }
  cplx x1 = cmk(0.0, 0.0), x2 = cmk(0.0, 0.0);
  // the lane's y~ of row i from its stage (packed real rows: the real part only)
  auto ytil = [&](const char *st, int i) -> cplx {
    const double *p = reinterpret_cast<const double *>(st + RING + 16 * lane);
    return i >= ipack ? ld2(p) : i >= i0 ? cmk(p[0], 0.0) : cmk(0.0, 0.0);
  };
  auto back_complex = [&](int i) {
    const char *st = begin(i);
    const double *row = reinterpret_cast<const double *>(st);
    cplx x = cfms(ytil(st, i), ld2(row + 4), x1);
    if (flag(st, i)) x = cfms(x, ld2(row + 6), x2);
    end_back(i);
    ystore(i, x);
    x2 = x1; x1 = x;
  };
  auto back_real = [&](int i) {
    const char *st = begin(i);
    const double *row = reinterpret_cast<const double *>(st);
    const cplx yi = ytil(st, i);
    const double u1 = row[CF ? 4 : 2];
    cplx x = cmk(fma(-u1, x1.re, yi.re), fma(-u1, x1.im, yi.im));
    if (flag(st, i)) {
      const double u2 = row[CF ? 6 : 3];
      x.re = fma(-u2, x2.re, x.re);
      x.im = fma(-u2, x2.im, x.im);
    }
    end_back(i);
    ystore(i, x);
    x2 = x1; x1 = x;
  };
  i = iend;
  if (CF) for (; i >= rhi; --i) back_complex(i);
  for (; i >= rlo; --i) back_real(i);
  if (CF) for (; i >= 0; --i) back_complex(i);
}

// Staging of the projection sweep: each warp owns TRI_STAGES stages of shared memory (2 or 4: a
// plan option the autotuner sets) and copies the operands of row i + TRI_STAGES while row i is
// swept. Forward stage: the table row (FSW doubles) and up to 4 ring values per lane
// ([slot][lane]); backward stage: table doubles 18..23 (u1, u2, swap flag) and the lane's y~.
template <bool CIN>
__host__ __device__ constexpr int tri_stage_bytes() { return FSW * 8 + 4 * 32 * (CIN ? 16 : 8); }
template <bool CIN, int TRI_STAGES>
__host__ __device__ constexpr int tri_smem_bytes() { return TRI_WARPS * TRI_STAGES * tri_stage_bytes<CIN>(); }

// The projection's sweep over the condensed, pivot-scaled table (plan: build_fs): rows
// i0 .. itop, y~ = y / d stored, so the back substitution is x = y~ - u1 x' - u2 x''. The rows
// with real entries [frlo, frhi) use real coefficients; while no complex value has entered the
// sweep (real densities and the run starts at i0) the forward recurrence is real.
// CD: complex mode-space data (complex AP or complex densities). sw: the warp's stages; the
// active lanes are 0 .. nact-1 (mask).
template <bool CD, bool CIN, int TRI_STAGES>
__device__ __forceinline__ void tri_fs_body(const Item &it, const SubDesc &d, const double *tab, double *ws, int b,
                                            int q, char *sw, int lane, int nact, unsigned mask) {
  constexpr int VS = CIN ? 16 : 8, SB = tri_stage_bytes<CIN>(), RING = FSW * 8;
  // descriptor fields in registers: the copies' memory clobbers would otherwise reload them
  const int i0 = d.i0, nfirst = d.nfirst, nlo = d.nlo, nhi = d.nhi, Nq = d.Nq, Ph = d.Ph;
  const bool xsym = d.xsym;
  const double *T = tab + d.fs_off + (long long)(q - 1) * d.NYf * FSW;
  const double *sg = tab + d.seg_off + 5 * (q - 1);
  const int frlo = (int)sg[2], frhi = (int)sg[3], itop = (int)sg[4];
  const int N2 = 2 * d.Nx;
  const double *S = tab + d.sin_off;
  const double sm0 = S[(q * d.mlo) % N2], sm1 = S[(q * (d.mlo + 1)) % N2];
  const double sm2 = S[(q * (d.mhi - 1)) % N2], sm3 = S[(q * d.mhi) % N2];
  const int par = (q & 1) ? 0 : 1;
  const double *r = ws + it.r_off;
  const double *gr = ws + it.gr_off;
  double *y = ws + it.y_off;
  const int nc = it.ncols, P = d.Px;
  const long long ybase = (long long)(q - 1) * d.NYf * nc + b;
  auto ystore = [&](int i, cplx v) {
    const long long o = ybase + (long long)(i - i0) * nc;
    if (CD) st2(y + 2 * o, v); else y[o] = v.re;
  };
  // complex data whose y~ is still real (the real forward run of real data): the warp's 32 real
  // values of row i packed into the first half of its 32 complex slots (lane's own column b), so
  // the round trip moves 8 bytes a value instead of 16. The back substitution stores the kept x
  // over them only after every lane's copy of row i has landed (the warp syncs first).
  auto ystore_re = [&](int i, double v) {
    if (CD) y[2 * (ybase + (long long)(i - i0) * nc) - lane] = v; else y[ybase + (long long)(i - i0) * nc] = v;
  };
  int ipack = i0;   // rows i0 .. ipack-1 hold packed real y~
  auto dense = [&](int n) -> int {
    return n == nlo ? 0 : n == nlo + 1 ? 1 : n == nhi - 1 ? 2 : n == nhi ? 3 : -1;
  };
  // ---- staging: forward rows
  auto fetch_fwd = [&](int i) {
    char *st = sw + ((i - i0) & (TRI_STAGES - 1)) * SB;
    const double *src = T + (long long)(i - i0) * FSW;
    if (nact >= FSW / 2) {
      if (lane < FSW / 2) cp_async16(st + 16 * lane, src + 2 * lane);
    } else {
      for (int c = lane; c < FSW / 2; c += nact) cp_async16(st + 16 * c, src + 2 * c);
    }
    const int n = i + 1 + nfirst;
    if (n >= nlo && n <= nhi) {
      char *rb = st + RING + VS * lane;
      auto cpv = [&](int slot, const double *base, long long o) {
        if (CIN) cp_async16(rb + slot * 32 * VS, base + 2 * o); else cp_async8(rb + slot * 32 * VS, base + o);
      };
      const int rr = dense(n);
      if (rr >= 0) {
        cpv(0, gr, ((long long)rr * Nq + (q - 1)) * nc + b);
      } else if (xsym) {
        const long long base = 8LL * Ph + 4 * (n - nlo - 2) + par;
        cpv(0, r, base * nc + b);
        cpv(1, r, (base + 2) * nc + b);
      } else {
        const long long ri = 2 * P + 4 * (n - nlo - 2);
        for (int s_ = 0; s_ < 4; ++s_) cpv(s_, r, (ri + s_) * nc + b);
      }
    }
    cp_async_commit();
  };
  // ring value `slot` of this lane in stage st
  auto sv = [&](const char *st, int slot) -> cplx {
    const double *p = reinterpret_cast<const double *>(st + RING + VS * lane + slot * 32 * VS);
    return CIN ? ld2(p) : cmk(p[0], 0.0);
  };
  // raw right-hand side of grid row n (swapped steps). Real data (basis columns, !CIN): only the
  // real part is formed; multiplying the zero imaginary parts would cost FP64 instructions that
  // the compiler cannot drop (0 x is not 0 for every x in IEEE arithmetic).
  auto graw = [&](const char *st, int n) -> cplx {
    if (n < nlo || n > nhi) return cmk(0.0, 0.0);
    if (dense(n) >= 0) return sv(st, 0);
    if (!CIN) {
      if (xsym) return cmk(fma(sm1, sv(st, 1).re, sm0 * sv(st, 0).re), 0.0);
      double v = sm0 * sv(st, 0).re;
      v = fma(sm1, sv(st, 1).re, v); v = fma(sm2, sv(st, 2).re, v); v = fma(sm3, sv(st, 3).re, v);
      return cmk(v, 0.0);
    }
    if (xsym) {
      const cplx a0 = sv(st, 0);
      return caxpy(sm1, sv(st, 1), cmk(sm0 * a0.re, sm0 * a0.im));
    }
    cplx v = cmk(0.0, 0.0);
    v = caxpy(sm0, sv(st, 0), v); v = caxpy(sm1, sv(st, 1), v); v = caxpy(sm2, sv(st, 2), v); v = caxpy(sm3, sv(st, 3), v);
    return v;
  };
  // scaled right-hand side g / d_{i+1} of grid row n from table row `row` (complex coefficients)
  auto ghat_c = [&](const char *st, const double *row, int n) -> cplx {
    if (n < nlo || n > nhi) return cmk(0.0, 0.0);
    const cplx sc = ld2(row + 8);
    if (dense(n) >= 0) {
      const cplx g = sv(st, 0);
      if (CIN) return cmul(sc, g);
      return cmk(sc.re * g.re, sc.im * g.re);
    }
    if (xsym) {
      if (CIN) return cadd(cmul(ld2(row + 10), sv(st, 0)), cmul(ld2(row + 12), sv(st, 1)));
      const double a0 = sv(st, 0).re, a1 = sv(st, 1).re;
      const cplx c0 = ld2(row + 10), c1 = ld2(row + 12);
      return cmk(fma(c1.re, a1, c0.re * a0), fma(c1.im, a1, c0.im * a0));
    }
    cplx v = cmk(0.0, 0.0);
    for (int s_ = 0; s_ < 4; ++s_) v = cadd(v, cmul(ld2(row + 10 + 2 * s_), sv(st, s_)));
    return v;
  };
  // the same with real coefficients (rows of the real run); real data: the real part only
  auto ghat_r = [&](const char *st, const double *row, int n) -> cplx {
    if (n < nlo || n > nhi) return cmk(0.0, 0.0);
    const double sc = row[8];
    if (dense(n) >= 0) {
      const cplx g = sv(st, 0);
      if (CIN) return cmk(sc * g.re, sc * g.im);
      return cmk(sc * g.re, 0.0);
    }
    if (!CIN) {
      if (xsym) return cmk(fma(row[12], sv(st, 1).re, row[10] * sv(st, 0).re), 0.0);
      double v = row[10] * sv(st, 0).re;
      for (int s_ = 1; s_ < 4; ++s_) v = fma(row[10 + 2 * s_], sv(st, s_).re, v);
      return cmk(v, 0.0);
    }
    if (xsym) {
      const cplx a0 = sv(st, 0);
      return caxpy(row[12], sv(st, 1), cmk(row[10] * a0.re, row[10] * a0.im));
    }
    cplx v = cmk(0.0, 0.0);
    for (int s_ = 0; s_ < 4; ++s_) v = caxpy(row[10 + 2 * s_], sv(st, s_), v);
    return v;
  };
  // the swap flag (0.0 or 1.0) tested on its bits: an integer compare, not an FP64-pipe DSETP
  auto swapped = [](double flag) { return __double_as_longlong(flag) != 0; };
  // stage of row i ready (this lane's copies complete, then every lane's visible)
  auto begin_fwd = [&](int i) -> const char * {
    cp_async_wait<TRI_STAGES - 1>();
    __syncwarp(mask);
    return sw + ((i - i0) & (TRI_STAGES - 1)) * SB;
  };
  // every lane is done with the stage of row i: refill it with row i + TRI_STAGES
  auto end_fwd = [&](int i) {
    __syncwarp(mask);
    if (i + TRI_STAGES < itop) fetch_fwd(i + TRI_STAGES); else cp_async_commit();
  };
  for (int j = 0; j < TRI_STAGES; ++j) {
    if (i0 + j < itop) fetch_fwd(i0 + j); else cp_async_commit();
  }
  // ---- forward sweep
  cplx ct = cmk(0.0, 0.0);
  int i = i0;
  if (CD) {
    for (; i < min(frlo, itop); ++i) {
      const char *st = begin_fwd(i);
      const double *row = reinterpret_cast<const double *>(st);
      const int n = i + 1 + nfirst;
      if (!swapped(row[22])) { ystore(i, ct); ct = cfms(ghat_c(st, row, n), ld2(row), ct); }
      else {
        const cplx g = graw(st, n);
        ystore(i, cmul(ld2(row + 6), g));
        ct = cfms(cmul(ld2(row + 2), ct), ld2(row + 4), g);
      }
      end_fwd(i);
    }
  }
  {
    const int e = min(max(frhi, i), itop);
    if (!CIN && i == i0) {     // real data so far: real recurrence
      for (; i < e; ++i) {
        const char *st = begin_fwd(i);
        const double *row = reinterpret_cast<const double *>(st);
        const int n = i + 1 + nfirst;
        if (!swapped(row[22])) { ystore_re(i, ct.re); ct.re = fma(-row[0], ct.re, ghat_r(st, row, n).re); }
        else {
          const double g = graw(st, n).re;
          ystore_re(i, row[6] * g);
          ct.re = fma(-row[4], g, row[2] * ct.re);
        }
        end_fwd(i);
      }
      ipack = i;
    } else {
      for (; i < e; ++i) {
        const char *st = begin_fwd(i);
        const double *row = reinterpret_cast<const double *>(st);
        const int n = i + 1 + nfirst;
        if (!swapped(row[22])) { ystore(i, ct); ct = caxpy(-row[0], ct, ghat_r(st, row, n)); }
        else {
          const cplx g = graw(st, n);
          ystore(i, cmk(row[6] * g.re, row[6] * g.im));
          ct = caxpy(-row[4], g, cmk(row[2] * ct.re, row[2] * ct.im));
        }
        end_fwd(i);
      }
    }
  }
  if (CD) {
    for (; i < itop; ++i) {
      const char *st = begin_fwd(i);
      const double *row = reinterpret_cast<const double *>(st);
      const int n = i + 1 + nfirst;
      if (!swapped(row[22])) { ystore(i, ct); ct = cfms(ghat_c(st, row, n), ld2(row), ct); }
      else {
        const cplx g = graw(st, n);
        ystore(i, cmul(ld2(row + 6), g));
        ct = cfms(cmul(ld2(row + 2), ct), ld2(row + 4), g);
      }
      end_fwd(i);
    }
  }
  ystore(itop, ct);
  // the stored y~ are read back below by this thread's asynchronous copies: order them after
  // its stores
  __threadfence_block();
  // ---- back substitution (rows nlo-1 .. nhi+1 are kept)
  auto fetch_back = [&](int i) {
    char *st = sw + ((itop - i) & (TRI_STAGES - 1)) * SB;
    const double *src = T + (long long)(i - i0) * FSW + 18;
    if (nact >= 3) {
      if (lane < 3) cp_async16(st + 16 * lane, src + 2 * lane);
    } else {
      for (int c = lane; c < 3; c += nact) cp_async16(st + 16 * c, src + 2 * c);
    }
    const long long o = ybase + (long long)(i - i0) * nc;
    if (!CD) cp_async8(st + RING + 8 * lane, y + o);
    else if (i < ipack) cp_async8(st + RING + 16 * lane, y + 2 * o - lane);
    else cp_async16(st + RING + 16 * lane, y + 2 * o);
    cp_async_commit();
  };
  for (int j = 0; j < TRI_STAGES; ++j) {
    if (itop - j >= i0) fetch_back(itop - j); else cp_async_commit();
  }
  const int ikeep = nhi + 1 - nfirst;
  cplx x1 = cmk(0.0, 0.0), x2 = cmk(0.0, 0.0);
  int emax = 0;   // largest biased exponent of the kept rows (integer compares only)
  auto bexp = [](double v) { return (__double2hiint(v) >> 20) & 0x7ff; };
  for (i = itop; i >= i0; --i) {
    cp_async_wait<TRI_STAGES - 1>();
    __syncwarp(mask);
    const char *st = sw + ((itop - i) & (TRI_STAGES - 1)) * SB;
    const double *rb = reinterpret_cast<const double *>(st);        // table doubles 18..23
    const double *yp = reinterpret_cast<const double *>(st + RING + (CD ? 16 : 8) * lane);
    const cplx yi = CD && i >= ipack ? ld2(yp) : cmk(yp[0], 0.0);
    cplx x;
    if (!CD || (i >= frlo && i < frhi)) {
      x = cmk(fma(-rb[0], x1.re, yi.re), CD ? fma(-rb[0], x1.im, yi.im) : 0.0);
      if (swapped(rb[4])) { x.re = fma(-rb[2], x2.re, x.re); if (CD) x.im = fma(-rb[2], x2.im, x.im); }
    } else {
      x = cfms(yi, ld2(rb), x1);
      if (swapped(rb[4])) x = cfms(x, ld2(rb + 2), x2);
    }
    __syncwarp(mask);
    if (i - TRI_STAGES >= i0) fetch_back(i - TRI_STAGES); else cp_async_commit();
    if (i <= ikeep) {
      ystore(i, x);
      emax = max(emax, max(bexp(x.re), bexp(x.im)));
    }
    x2 = x1; x1 = x;
  }
  // per column, over every mode: the common power-of-two scale of the tensor-core gamma columns
  if (d.tc_cols) atomicMax(reinterpret_cast<int *>(ws + it.red_off) + b, emax);
}

template <bool CIN, bool FULL, int TRI_STAGES>
__global__ void __launch_bounds__(32 * TRI_WARPS, 32 / TRI_WARPS) k_tri(Batch bt, const SubDesc *subs, const double *tab, const uint8_t *pivtab,
                                             double *ws) {
  Item it; int local;
  locate(bt, bt.order ? bt.order[blockIdx.x] : (int)blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_TRI);
  const SubDesc &d = subs[it.sub];
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int q = (local / cb) * TRI_WARPS + threadIdx.y + 1;
  // a warp shares q; its active lanes (columns b < ncols) are lanes 0 .. nact-1
  extern __shared__ __align__(16) char tri_sm[];
  const bool act = b < it.ncols && q <= d.Nq;
  const unsigned mask = __ballot_sync(0xffffffffu, act);
  if (!act) return;
  if (FULL) {
    char *sw = tri_sm + threadIdx.y * 2 * full_stage_bytes<CIN>();
    if (d.cplx) tri_full_body<true, CIN>(it, d, tab, pivtab, ws, b, q, sw, threadIdx.x, __popc(mask), mask);
    else tri_full_body<false, CIN>(it, d, tab, pivtab, ws, b, q, sw, threadIdx.x, __popc(mask), mask);
  } else {
    char *sw = tri_sm + threadIdx.y * TRI_STAGES * tri_stage_bytes<CIN>();
    if (d.cplx || CIN) tri_fs_body<true, CIN, TRI_STAGES>(it, d, tab, ws, b, q, sw, threadIdx.x, __popc(mask), mask);
    else tri_fs_body<false, CIN, TRI_STAGES>(it, d, tab, ws, b, q, sw, threadIdx.x, __popc(mask), mask);
  }
}

// ---------------------------------------------------------------- inverse transforms on gamma
template <bool CD, bool CIN>
__device__ __forceinline__ void write_out(const SubDesc &d, const Item &it, const double *ws, const double *tab,
                                          const double2 *xi_user, double2 *out, int kind, int b, int g, cplx u) {
  if (MDP_CHECKED && (g < 0 || g >= d.G || b < 0 || b >= it.ncols)) { flag_bounds(d.dstatus); return; }
  cplx v = cmk(-u.re, -u.im);
  if (kind == MDP_OUT_P) v = cadd(v, density<CIN>(d, it, ws, tab, xi_user, b, g));
  out[it.io_off + (long long)b * d.G + g] = make_double2(v.re, v.im);
}

// u(m, n) = (2/Nx) sum_q sin(pi q m/Nx) yhat(q, n) for the 4 full gamma rows. Centred
// subdomains: one thread gives u(m) = E + O and u(Nx - m) = E - O from the odd-q (E) and
// even-q (O) partial sums, since sin(pi q (Nx-m)/Nx) = (-1)^(q+1) sin(pi q m/Nx).
template <bool CD, bool CIN>
__device__ __forceinline__ void inv_rows_body(const Item &it, const SubDesc &d, const double *tab, const double *ws,
                                              const double2 *xi_user, double2 *out, int kind, int b, int task) {
  const int W = d.Px + 2, Mr = d.Py - 2;
  const int span = d.xsym ? d.Ph + 1 : W;
  const int grow = task / span, dm = task % span, m = d.mlo - 1 + dm;
  const int n = grow == 0 ? d.nlo - 1 : grow == 1 ? d.nlo : grow == 2 ? d.nhi : d.nhi + 1;
  const int yrow = n - (d.nlo - 1);
  const double *Si = tab + d.sin_off + 2 * d.Nx;
  const int N2 = 2 * d.Nx;
  const double *y = ws + it.y_off;
  const long long qstride = (long long)d.NYf * it.ncols;
  const long long base = (long long)yrow * it.ncols + b;
  auto yv = [&](int q) -> cplx {
    const long long o = base + (long long)(q - 1) * qstride;
    return CD ? ld2(y + 2 * o) : cmk(y[o], 0.0);
  };
  cplx e = cmk(0.0, 0.0), o = cmk(0.0, 0.0);
  int j = m % N2;
  int q = 1;
  for (; q + 1 <= d.Nq; q += 2) {  // (odd, even) mode pairs
    const cplx v1 = yv(q), v2 = yv(q + 1);
    const double s1 = Si[j];
    j += m; if (j >= N2) j -= N2;
    const double s2 = Si[j];
    j += m; if (j >= N2) j -= N2;
    if (CD) { e = caxpy(s1, v1, e); o = caxpy(s2, v2, o); }
    else { e.re = fma(s1, v1.re, e.re); o.re = fma(s2, v2.re, o.re); }
  }
  if (q <= d.Nq) {
    const cplx v1 = yv(q);
    if (CD) e = caxpy(Si[j], v1, e); else e.re = fma(Si[j], v1.re, e.re);
  }
  auto gidx = [&](int mm) { const int k = mm - (d.mlo - 1); return grow <= 1 ? grow * W + k : 2 * W + 4 * Mr + (grow - 2) * W + k; };
  write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b, gidx(m), cadd(e, o));
  if (d.xsym && d.Nx - m != m) write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b, gidx(d.Nx - m), csub(e, o));
}

// The same rows by FFT: u(m) = (2/Nx) F_m with F the DST-I of yhat (dst1_post: one complex FFT
// of length Nx of the twisted sequence, radix-2 decimation in time in shared memory, inputs
// stored bit-reversed). One block: one gamma row and fpb = 1024/(2Nx) columns (or one column
// when Nx >= 512); the transforms take the first fpb Nx values of shared memory, the outputs the
// next fpb Nx.
template <bool CD, bool CIN>
__device__ __forceinline__ void inv_rows_fft_body(const Item &it, const SubDesc &d, const double *tab,
                                                  const double *ws, const double2 *xi_user, double2 *out, int kind,
                                                  int local, double2 *sm) {
  __shared__ double2 tot[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int grow = local & 3, cblk = local >> 2;
  const int b0 = cblk * d.fpb, nf = min(d.fpb, it.ncols - b0);
  const int N = d.Nx, H = N / 2;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  const double *sn = tab + d.sin_off;
  const int n = grow == 0 ? d.nlo - 1 : grow == 1 ? d.nlo : grow == 2 ? d.nhi : d.nhi + 1;
  const int yrow = n - (d.nlo - 1);
  const double *y = ws + it.y_off;
  const long long qstride = (long long)d.NYf * it.ncols;
  auto yv = [&](int q, int f) -> cplx {   // yhat(q) of column b0 + f, q = 1 .. N-1
    const long long o = (long long)(q - 1) * qstride + (long long)yrow * it.ncols + b0 + f;
    return CD ? ld2(y + 2 * o) : cmk(y[o], 0.0);
  };
  // the twisted sequence, bit-reversed, for the pairs (q, N - q); the column is fastest
  for (int idx = tid; idx < d.fpb * (H + 1); idx += nt) {
    const int f = idx % d.fpb, j = idx / d.fpb;
    double2 *S = sm + (long long)f * N;
    if (j == 0) { S[0] = make_double2(0.0, 0.0); continue; }
    cplx xa = cmk(0.0, 0.0), xb = cmk(0.0, 0.0);
    if (f < nf) {
      xa = yv(j, f);
      if (2 * j != N) xb = yv(N - j, f);
    }
    if (2 * j == N) { S[brev_lg(j, lg)] = make_double2(2.0 * xa.re, 2.0 * xa.im); continue; }
    cplx ya, yb;
    dst1_twist(xa, xb, sn[j], ya, yb);
    S[brev_lg(j, lg)] = make_double2(ya.re, ya.im);
    S[brev_lg(N - j, lg)] = make_double2(yb.re, yb.im);
  }
  __syncthreads();
  fft_r2_stages(sm, d.fpb, N, lg, sn);
  double2 *F = sm + (long long)d.fpb * N;
  dst1_post(sm, F, d.fpb, N, tot);
  const int W = d.Px + 2, Mr = d.Py - 2;
  const double sc = 2.0 / N;
  for (int idx = tid; idx < nf * W; idx += nt) {
    const int f = idx / W, dm = idx % W, m = d.mlo - 1 + dm;
    const double2 V = F[(long long)f * N + m];
    const cplx u = cmk(sc * V.x, sc * V.y);
    const int g = grow <= 1 ? grow * W + dm : 2 * W + 4 * Mr + (grow - 2) * W + dm;
    write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b0 + f, g, u);
  }
}

template <bool CIN>
__global__ void __launch_bounds__(256) k_inv_rows(Batch bt, const SubDesc *subs, const double *tab, const double *ws,
                                                  const double2 *xi_user, double2 *out, int kind) {
  extern __shared__ double2 fft_sm[];
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_IROWS);
  const SubDesc &d = subs[it.sub];
  if (d.rows_fft) {
    if (d.cplx || CIN) inv_rows_fft_body<true, CIN>(it, d, tab, ws, xi_user, out, kind, local, fft_sm);
    else inv_rows_fft_body<false, CIN>(it, d, tab, ws, xi_user, out, kind, local, fft_sm);
    return;
  }
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int task = (local / cb) * 8 + threadIdx.y;
  if (b >= it.ncols || task >= 4 * (d.xsym ? d.Ph + 1 : d.Px + 2)) return;
  if (d.cplx || CIN) inv_rows_body<true, CIN>(it, d, tab, ws, xi_user, out, kind, b, task);
  else inv_rows_body<false, CIN>(it, d, tab, ws, xi_user, out, kind, b, task);
}

// the 4 gamma columns (mlo-1, mlo, mhi, mhi+1) of the middle rows nlo+1 .. nhi-1; centred
// subdomains pair mlo-1 with mhi+1 and mlo with mhi (odd-q / even-q partial sums)
template <bool CD, bool CIN>
__device__ __forceinline__ void inv_cols_body(const Item &it, const SubDesc &d, const double *tab, const double *ws,
                                              const double2 *xi_user, double2 *out, int kind, int b, int t) {
  const int yrow = t + 2;  // n = nlo + 1 + t
  const double *Si = tab + d.sin_off + 2 * d.Nx;
  const int N2 = 2 * d.Nx;
  const double *y = ws + it.y_off;
  const long long qstride = (long long)d.NYf * it.ncols;
  const long long base = (long long)yrow * it.ncols + b;
  const int W = d.Px + 2;
  auto yv = [&](int q) -> cplx {
    const long long o = base + (long long)(q - 1) * qstride;
    return CD ? ld2(y + 2 * o) : cmk(y[o], 0.0);
  };
  if (d.xsym) {
    const int m0 = d.mlo - 1, m1 = d.mlo;
    int j0 = m0 % N2, j1 = m1 % N2;
    cplx e0 = cmk(0, 0), o0 = cmk(0, 0), e1 = cmk(0, 0), o1 = cmk(0, 0);
    int q = 1;
    for (; q + 1 <= d.Nq; q += 2) {
      const cplx va = yv(q), vb = yv(q + 1);
      const double a0 = Si[j0], a1 = Si[j1];
      j0 += m0; if (j0 >= N2) j0 -= N2;
      j1 += m1; if (j1 >= N2) j1 -= N2;
      const double b0 = Si[j0], b1 = Si[j1];
      j0 += m0; if (j0 >= N2) j0 -= N2;
      j1 += m1; if (j1 >= N2) j1 -= N2;
      if (CD) { e0 = caxpy(a0, va, e0); e1 = caxpy(a1, va, e1); o0 = caxpy(b0, vb, o0); o1 = caxpy(b1, vb, o1); }
      else {
        e0.re = fma(a0, va.re, e0.re); e1.re = fma(a1, va.re, e1.re);
        o0.re = fma(b0, vb.re, o0.re); o1.re = fma(b1, vb.re, o1.re);
      }
    }
    if (q <= d.Nq) {
      const cplx va = yv(q);
      if (CD) { e0 = caxpy(Si[j0], va, e0); e1 = caxpy(Si[j1], va, e1); }
      else { e0.re = fma(Si[j0], va.re, e0.re); e1.re = fma(Si[j1], va.re, e1.re); }
    }
    const int g0 = 2 * W + 4 * t;
    write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b, g0 + 0, cadd(e0, o0));
    write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b, g0 + 1, cadd(e1, o1));
    write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b, g0 + 2, csub(e1, o1));
    write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b, g0 + 3, csub(e0, o0));
    return;
  }
  const int ms[4] = {d.mlo - 1, d.mlo, d.mhi, d.mhi + 1};
  int j[4] = {ms[0] % N2, ms[1] % N2, ms[2] % N2, ms[3] % N2};
  cplx acc[4] = {cmk(0, 0), cmk(0, 0), cmk(0, 0), cmk(0, 0)};
  for (int q = 1; q <= d.Nq; ++q) {
    const cplx v = yv(q);
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const double sv = Si[j[s]];
      if (CD) acc[s] = caxpy(sv, v, acc[s]); else acc[s].re = fma(sv, v.re, acc[s].re);
      j[s] += ms[s];
      if (j[s] >= N2) j[s] -= N2;
    }
  }
#pragma unroll
  for (int s = 0; s < 4; ++s)
    write_out<CD, CIN>(d, it, ws, tab, xi_user, out, kind, b, 2 * W + 4 * t + s, acc[s]);
}

template <bool CIN>
__global__ void __launch_bounds__(256) k_inv_cols(Batch bt, const SubDesc *subs, const double *tab, const double *ws,
                                                  const double2 *xi_user, double2 *out, int kind) {
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_ICOLS);
  const SubDesc &d = subs[it.sub];
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int t = (local / cb) * 8 + threadIdx.y;
  if (b >= it.ncols || t >= d.Py - 2) return;
  if (d.cplx || CIN) inv_cols_body<true, CIN>(it, d, tab, ws, xi_user, out, kind, b, t);
  else inv_cols_body<false, CIN>(it, d, tab, ws, xi_user, out, kind, b, t);
}

// ---------------------------------------------------------------- receivers
// P_N+ xi at the receiver row nrec, nodes m = mlo+1 .. mhi-1 (not on gamma, so w = 0 there and
// the difference potential is -G^(h) r): u = -(2/Nx) sum_q sin(pi q m/Nx) yhat(q, nrec).
// Output out_rec[rec_off + c * (Px - 2) + (m - mlo - 1)]; centred subdomains give m and Nx - m.
template <bool CD>
__device__ __forceinline__ void inv_rec_body(const Item &it, const SubDesc &d, const double *tab, const double *ws,
                                             double2 *out_rec, int b, int task) {
  const int m = d.mlo + 1 + task;
  const int yrow = d.nrec - (d.nlo - 1);
  const double *Si = tab + d.sin_off + 2 * d.Nx;
  const int N2 = 2 * d.Nx;
  const double *y = ws + it.y_off;
  const long long qstride = (long long)d.NYf * it.ncols;
  const long long base = (long long)yrow * it.ncols + b;
  auto yv = [&](int q) -> cplx {
    const long long o = base + (long long)(q - 1) * qstride;
    return CD ? ld2(y + 2 * o) : cmk(y[o], 0.0);
  };
  cplx e = cmk(0.0, 0.0), o = cmk(0.0, 0.0);
  int j = m % N2;
  int q = 1;
  for (; q + 1 <= d.Nq; q += 2) {
    const cplx v1 = yv(q), v2 = yv(q + 1);
    const double s1 = Si[j];
    j += m; if (j >= N2) j -= N2;
    const double s2 = Si[j];
    j += m; if (j >= N2) j -= N2;
    e = caxpy(s1, v1, e);
    o = caxpy(s2, v2, o);
  }
  if (q <= d.Nq) e = caxpy(Si[j], yv(q), e);
  const long long col = (long long)(it.col0 + b) * (d.Px - 2);
  if (d.xsym) {
    const cplx up = cadd(e, o), um = csub(e, o);
    out_rec[d.rec_off + col + (m - d.mlo - 1)] = make_double2(-up.re, -up.im);
    if (d.Nx - m != m) out_rec[d.rec_off + col + (d.Nx - m - d.mlo - 1)] = make_double2(-um.re, -um.im);
  } else {
    const cplx u = cadd(e, o);
    out_rec[d.rec_off + col + (m - d.mlo - 1)] = make_double2(-u.re, -u.im);
  }
}

__global__ void __launch_bounds__(256) k_inv_rec(Batch bt, const SubDesc *subs, const double *tab, const double *ws,
                                                 double2 *out_rec, int cd) {
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_IREC);
  const SubDesc &d = subs[it.sub];
  if (d.nrec < 0) return;
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int task = (local / cb) * 8 + threadIdx.y;
  if (b >= it.ncols || task >= (d.xsym ? d.Ph - 1 : d.Px - 2)) return;
  if (d.cplx || cd) inv_rec_body<true>(it, d, tab, ws, out_rec, b, task);
  else inv_rec_body<false>(it, d, tab, ws, out_rec, b, task);
}

// ---------------------------------------------------------------- full-grid solves
// u = G^(h) g or A^{-H} g on the whole grid (test and reconstruction primitive). Mode-space
// buffer buf[r][q-1][i] (complex), i = matrix row of the y unknowns.

// Solve T_q z = b (adjoint = 0) or T_q^H z = b (adjoint = 1) in place on a contiguous vector.
template <bool CF>
__device__ void mode_solve_inplace(const double *F, const uint8_t *pv, int N, double *z, int adjoint) {
  constexpr int FW = CF ? 8 : 4;
  auto fl = [&](int i, int w) -> cplx { return CF ? ld2(F + i * FW + 2 * w) : cmk(F[i * FW + w], 0.0); };
  auto cj = [](cplx a) { return cmk(a.re, -a.im); };
  if (!adjoint) {
    cplx cur = ld2(z);
    for (int i = 0; i < N - 1; ++i) {
      const cplx g = ld2(z + 2 * (i + 1));
      const cplx l = fl(i, 0);
      cplx yv;
      if (pv[i]) { yv = g; cur = cfms(cur, l, g); } else { yv = cur; cur = cfms(g, l, cur); }
      st2(z + 2 * i, yv);
    }
    st2(z + 2 * (N - 1), cur);
    cplx x1 = cmk(0, 0), x2 = cmk(0, 0);
    for (int i = N - 1; i >= 0; --i) {
      cplx x = cfms(cmul(fl(i, 1), ld2(z + 2 * i)), fl(i, 2), x1);
      if (pv[i]) x = cfms(x, fl(i, 3), x2);
      st2(z + 2 * i, x);
      x2 = x1; x1 = x;
    }
  } else {
    // U^H zt = b with zt_i = conj(d_i) z_i, then z = P_0 E_0^H ... P_{N-2} E_{N-2}^H z
    cplx t1 = cmk(0, 0), t2 = cmk(0, 0);
    for (int i = 0; i < N; ++i) {
      cplx v = ld2(z + 2 * i);
      if (i >= 1) v = cfms(v, cj(fl(i - 1, 2)), t1);
      if (i >= 2 && pv[i - 2]) v = cfms(v, cj(fl(i - 2, 3)), t2);
      st2(z + 2 * i, cmul(cj(fl(i, 1)), v));
      t2 = t1; t1 = v;
    }
    // `up` is the current value at position i+1; after step i position i+1 is final
    cplx up = ld2(z + 2 * (N - 1));
    for (int i = N - 2; i >= 0; --i) {
      const cplx zi = cfms(ld2(z + 2 * i), cj(fl(i, 0)), up);
      if (pv[i]) st2(z + 2 * (i + 1), zi);          // swap: i+1 takes the update, i keeps `up`
      else { st2(z + 2 * (i + 1), up); up = zi; }
    }
    st2(z, up);
  }
}

__global__ void k_full_fwd(const SubDesc *subs, int sub, const double *tab, const double2 *g, double *buf,
                           int r0, int nr, int adjoint) {
  const SubDesc &d = subs[sub];
  const int q = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int i = blockIdx.y;
  const int rl = blockIdx.z;
  if (q > d.Nq || rl >= nr) return;
  const int n = i + d.nfirst;
  cplx acc = cmk(0.0, 0.0);
  const bool interior = n >= 1 && n <= d.ny - 2;
  if (interior || adjoint) {
    const double *S = tab + d.sin_off;
    const int N2 = 2 * d.Nx;
    const double2 *row = g + ((long long)(r0 + rl) * d.ny + n) * d.nx;
    int j = q;
    for (int m = 1; m <= d.Nx - 1; ++m) {
      const double2 v = row[m];
      acc = caxpy(S[j], cmk(v.x, v.y), acc);
      j += q;
      if (j >= N2) j -= N2;
    }
  }
  st2(buf + 2 * (((long long)rl * d.Nq + (q - 1)) * d.Nt + i), acc);
}

__global__ void k_full_tri(const SubDesc *subs, int sub, const double *tab, const uint8_t *pivtab, double *buf,
                           int nr, int adjoint) {
  const SubDesc &d = subs[sub];
  const int q = blockIdx.x * blockDim.x + threadIdx.x + 1;
  const int rl = blockIdx.y;
  if (q > d.Nq || rl >= nr) return;
  double *z = buf + 2 * (((long long)rl * d.Nq + (q - 1)) * d.Nt);
  const uint8_t *pv = pivtab + d.piv_off + (long long)(q - 1) * d.Nt;
  if (d.cplx) mode_solve_inplace<true>(tab + d.fact_off + (long long)(q - 1) * d.Nt * 8, pv, d.Nt, z, adjoint);
  else mode_solve_inplace<false>(tab + d.fact_off + (long long)(q - 1) * d.Nt * 4, pv, d.Nt, z, adjoint);
}

__global__ void k_full_inv(const SubDesc *subs, int sub, const double *tab, const double *buf, double2 *u,
                           int r0, int nr, int adjoint) {
  const SubDesc &d = subs[sub];
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = blockIdx.y;
  const int rl = blockIdx.z;
  if (m >= d.nx || rl >= nr) return;
  const int i = n - d.nfirst;
  cplx acc = cmk(0.0, 0.0);
  if (m >= 1 && m <= d.Nx - 1 && i >= 0 && i < d.Nt) {
    const double *Si = tab + d.sin_off + 2 * d.Nx;
    const int N2 = 2 * d.Nx;
    int j = m;
    const double *col = buf + 2 * ((long long)rl * d.Nq * d.Nt + i);
    for (int q = 1; q <= d.Nq; ++q) {
      acc = caxpy(Si[j], ld2(col + 2 * (long long)(q - 1) * d.Nt), acc);
      j += m;
      if (j >= N2) j -= N2;
    }
    // A^{-H} of the unscaled AP: the Sommerfeld rows of T_q carry a 1/h row scale
    if (adjoint && d.cplx && (n == 0 || n == d.ny - 1)) { acc.re /= d.h; acc.im /= d.h; }
  }
  u[((long long)(r0 + rl) * d.ny + n) * d.nx + m] = make_double2(acc.re, acc.im);
}

cudaError_t launch_solve(const mdp_plan *p, int sub, int nrhs, const double2 *g, double2 *u, int adjoint,
                         cudaStream_t st) {
  const SubDesc &d = p->subs[sub].d;
  const long long per = (long long)d.Nq * d.Nt * 2;
  long long chunk = p->ws_doubles / per;
  if (chunk < 1) return cudaErrorMemoryAllocation;
  if (chunk > 65535) chunk = 65535;
  for (int r0 = 0; r0 < nrhs; r0 += (int)chunk) {
    const int nr = (int)std::min<long long>(chunk, nrhs - r0);
    k_full_fwd<<<dim3((d.Nq + 63) / 64, d.Nt, nr), 64, 0, st>>>(p->d_subs, sub, p->d_tables, g, p->d_ws, r0, nr, adjoint);
    k_full_tri<<<dim3((d.Nq + 63) / 64, nr), 64, 0, st>>>(p->d_subs, sub, p->d_tables, p->d_piv, p->d_ws, nr, adjoint);
    k_full_inv<<<dim3((d.nx + 63) / 64, d.ny, nr), 64, 0, st>>>(p->d_subs, sub, p->d_tables, p->d_ws, u, r0, nr, adjoint);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- potential on the grid
// The extended basis densities xi_c on gamma (k_extend's values, zero where the node belongs
// to another side than the column's), out[c][g] complex, for the item's columns.
__global__ void __launch_bounds__(256) k_basis_out(Item it, const SubDesc *subs, const double *tab, const double *ws,
                                                   double2 *out) {
  const SubDesc &d = subs[it.sub];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)it.ncols * d.G) return;
  const int b = (int)(t / d.G), g = (int)(t % d.G);
  const cplx v = density<false>(d, it, ws, tab, nullptr, b, g);
  out[(long long)b * d.G + g] = make_double2(v.re, v.im);
}

// Right-hand side of the potential: r = L^(h) w on the ring inside M+ (w = xi on gamma, 0
// elsewhere: the only nodes of M+ where L w is nonzero), written into the zeroed grid
// u[c][n][m] that the full-grid solve then reads.
__global__ void __launch_bounds__(256) k_pot_rhs(int sub, const SubDesc *subs, int ncols, const double2 *xi, double2 *u) {
  const SubDesc &d = subs[sub];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ncols * d.R) return;
  const int c = (int)(t / d.R), ri = (int)(t % d.R);
  int n, m;
  ring_node(d, ri, n, m);
  const double2 *x = xi + (long long)c * d.G;
  cplx acc = cmk(0.0, 0.0);
#pragma unroll
  for (int dn = -1; dn <= 1; ++dn) {
#pragma unroll
    for (int dm = -1; dm <= 1; ++dm) {
      const int g = gamma_index(d, n + dn, m + dm);
      if (g < 0) continue;
      const int nb = (dn != 0) + (dm != 0);
      const double cf = nb == 0 ? d.c0 : nb == 1 ? d.c1 : d.c2;
      acc = caxpy(cf, cmk(x[g].x, x[g].y), acc);
    }
  }
  u[((long long)c * d.ny + n) * d.nx + m] = make_double2(acc.re, acc.im);
}

// u <- w - u on every node (w = xi on gamma, 0 elsewhere): the difference potential.
__global__ void __launch_bounds__(256) k_pot_fix(int sub, const SubDesc *subs, int ncols, const double2 *xi, double2 *u) {
  const SubDesc &d = subs[sub];
  const long long npt = (long long)d.nx * d.ny;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)ncols * npt) return;
  const int c = (int)(t / npt);
  const long long k = t % npt;
  const int n = (int)(k / d.nx), m = (int)(k % d.nx);
  double2 v = u[t];
  v.x = -v.x; v.y = -v.y;
  const int g = gamma_index(d, n, m);
  if (g >= 0) { const double2 w = xi[(long long)c * d.G + g]; v.x += w.x; v.y += w.y; }
  u[t] = v;
}

// ---------------------------------------------------------------- source terms
// Ex^(I) f on gamma (the source terms of the equation-based extension): from the foot data
// src4[g] = (f, d_n f, d_nn f, d_tt f) and the node's distance rho to its owner side,
// rho^2/2 f + rho^3/6 d_n f + rho^4/24 (d_nn f - d_tt f - k^2 f).
__global__ void __launch_bounds__(256) k_ext_source(int sub, const SubDesc *subs, const double *tab,
                                                    const double2 *src4, double2 *xi) {
  const SubDesc &d = subs[sub];
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d.G) return;
  const double rho = tab[d.geo_off + 4 * g + 2];
  const double r2 = 0.5 * rho * rho, r3 = r2 * rho / 3.0, r4 = r2 * r2 / 6.0;
  const double2 f = src4[4 * g], fn = src4[4 * g + 1], fnn = src4[4 * g + 2], ftt = src4[4 * g + 3];
  const double k2 = d.k * d.k;
  const double t4r = fnn.x - ftt.x - k2 * f.x, t4i = fnn.y - ftt.y - k2 * f.y;
  xi[g] = make_double2(fma(r4, t4r, fma(r3, fn.x, r2 * f.x)), fma(r4, t4i, fma(r3, fn.y, r2 * f.y)));
}

// g = (B^(h) f)|M+: f + (f_{m+1} + f_{m-1} + f_{n+1} + f_{n-1} - 4 f) / 12 on the nodes of M+
// (the rectangle mlo..mhi x nlo..nhi), 0 elsewhere.
__global__ void __launch_bounds__(256) k_apply_B(int sub, const SubDesc *subs, const double2 *f, double2 *g) {
  const SubDesc &d = subs[sub];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nx * d.ny) return;
  const int n = (int)(t / d.nx), m = (int)(t % d.nx);
  double2 v = make_double2(0.0, 0.0);
  if (m >= d.mlo && m <= d.mhi && n >= d.nlo && n <= d.nhi) {
    const double2 c = f[t], e = f[t + 1], w = f[t - 1], nn = f[t + d.nx], s = f[t - d.nx];
    v.x = c.x + (e.x + w.x + nn.x + s.x - 4.0 * c.x) / 12.0;
    v.y = c.y + (e.y + w.y + nn.y + s.y - 4.0 * c.y) / 12.0;
  }
  g[t] = v;
}

// F <- -F - Tr(ub) on gamma, u <- u + ub on the grid.
__global__ void __launch_bounds__(256) k_src_fin(int sub, const SubDesc *subs, const double2 *ub, double2 *F,
                                                 double2 *u) {
  const SubDesc &d = subs[sub];
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)d.nx * d.ny) return;
  const int n = (int)(t / d.nx), m = (int)(t % d.nx);
  const double2 b = ub[t];
  double2 v = u[t];
  v.x += b.x; v.y += b.y;
  u[t] = v;
  const int g = gamma_index(d, n, m);
  if (g >= 0) { const double2 q = F[g]; F[g] = make_double2(-q.x - b.x, -q.y - b.y); }
}

// Full-grid solve on caller-provided device tables and scratch (one subdomain at d_sub[0]).
cudaError_t launch_solve_raw(const SubDesc *d_sub, const SubDesc &hd, const double *tab, const uint8_t *piv,
                             double *buf, long long buf_doubles, int nrhs, const double2 *g, double2 *u, int adjoint,
                             cudaStream_t st) {
  const long long per = (long long)hd.Nq * hd.Nt * 2;
  long long chunk = buf_doubles / per;
  if (chunk < 1) return cudaErrorInvalidValue;
  if (chunk > 65535) chunk = 65535;
  for (int r0 = 0; r0 < nrhs; r0 += (int)chunk) {
    const int nr = (int)std::min<long long>(chunk, nrhs - r0);
    k_full_fwd<<<dim3((hd.Nq + 63) / 64, hd.Nt, nr), 64, 0, st>>>(d_sub, 0, tab, g, buf, r0, nr, adjoint);
    k_full_tri<<<dim3((hd.Nq + 63) / 64, nr), 64, 0, st>>>(d_sub, 0, tab, piv, buf, nr, adjoint);
    k_full_inv<<<dim3((hd.nx + 63) / 64, hd.ny, nr), 64, 0, st>>>(d_sub, 0, tab, buf, u, r0, nr, adjoint);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// P_N+ xi on the whole grid of subdomain `sub` for ncols densities (Eq. Potential_def):
// w - G^(h) (L^(h) w)|M+. u doubles as the right-hand side of the full-grid solve.
cudaError_t launch_potential(const mdp_plan *p, int sub, int ncols, const double2 *xi, double2 *u, cudaStream_t st) {
  const SubDesc &d = p->subs[sub].d;
  const long long npt = (long long)d.nx * d.ny;
  cudaError_t e = cudaMemsetAsync(u, 0, (size_t)ncols * npt * sizeof(double2), st);
  if (e != cudaSuccess) return e;
  const long long nr = (long long)ncols * d.R;
  k_pot_rhs<<<(unsigned)((nr + 255) / 256), 256, 0, st>>>(sub, p->d_subs, ncols, xi, u);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_solve(p, sub, ncols, u, u, 0, st);
  if (e != cudaSuccess) return e;
  const long long nt = (long long)ncols * npt;
  k_pot_fix<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(sub, p->d_subs, ncols, xi, u);
  return cudaGetLastError();
}

// The source's terms for subdomain `sub` (f on the grid, foot data src4 on gamma):
// F = -(P_gamma - I) Ex^(I) f - Tr G (B f)|M+ and u = P_N+ Ex^(I) f + G (B f)|M+ on the grid.
// Scratch at the top of the workspace: xi_I [G] and the grid of G (B f)|M+; the solves and the
// one-column projection use the workspace from its start.
cudaError_t launch_source_terms(mdp_plan *p, int sub, const double2 *f, const double2 *src4, double2 *F, double2 *u,
                                cudaStream_t st) {
  const SubDesc &d = p->subs[sub].d;
  const long long npt = (long long)d.nx * d.ny;
  const long long scratch = 2LL * d.G + 2 * npt + 64;
  long long xo, ro, go, yo, ao, so, reo, tot;
  item_workspace(d, 1, false, xo, ro, go, yo, ao, so, reo, tot);
  const long long need = std::max((long long)d.Nq * d.Nt * 2, tot) + scratch;
  if (p->ws_doubles < need) return cudaErrorMemoryAllocation;
  const long long top = (p->ws_doubles - scratch) & ~31LL;
  double2 *xi_i = reinterpret_cast<double2 *>(p->d_ws + top);
  double2 *ub = reinterpret_cast<double2 *>(p->d_ws + top + ((2LL * d.G + 31) & ~31LL));
  k_ext_source<<<(d.G + 255) / 256, 256, 0, st>>>(sub, p->d_subs, p->d_tables, src4, xi_i);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_potential(p, sub, 1, xi_i, u, st);                 // u = P_N+ Ex^(I) f
  if (e != cudaSuccess) return e;
  k_apply_B<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(sub, p->d_subs, f, ub);
  e = launch_solve(p, sub, 1, ub, ub, 0, st);                   // ub = G (B f)|M+
  if (e != cudaSuccess) return e;
  Item it;                                                       // F = (P_gamma - I) xi_I
  std::memset(&it, 0, sizeof it);
  it.sub = sub; it.col0 = 0; it.ncols = 1;
  it.xi_off = xo; it.r_off = ro; it.gr_off = go; it.y_off = yo; it.a_off = ao; it.s_off = so; it.red_off = reo;
  Batch fb[NFAM];
  for (int f_ = 0; f_ < NFAM; ++f_) {
    std::memset(&fb[f_], 0, sizeof fb[f_]);
    fb[f_].n_items = 1; fb[f_].one = it; fb[f_].total_blocks = blocks_for((Fam)f_, d, 1);
    set_bounds(p, fb[f_], d.G, false);
  }
  e = launch_project(p, fb, MDP_OUT_Q, xi_i, F, nullptr, st);
  if (e != cudaSuccess) return e;
  k_src_fin<<<(unsigned)((npt + 255) / 256), 256, 0, st>>>(sub, p->d_subs, ub, F, u);
  return cudaGetLastError();
}

// The extended basis densities of columns col0 .. col0+ncols-1 of subdomain `sub`, out[c][g].
cudaError_t launch_basis_densities(const mdp_plan *p, int sub, int col0, int ncols, double2 *out, cudaStream_t st) {
  const SubDesc &d = p->subs[sub].d;
  for (int c = 0; c < ncols; c += p->tile_cols) {
    Item it;
    std::memset(&it, 0, sizeof it);
    it.sub = sub; it.col0 = col0 + c; it.ncols = std::min(p->tile_cols, ncols - c);
    long long xo, ro, go, yo, ao, so, reo, tot;
    item_workspace(d, it.ncols, false, xo, ro, go, yo, ao, so, reo, tot);
    it.xi_off = xo; it.r_off = ro; it.gr_off = go; it.y_off = yo; it.a_off = ao; it.s_off = so; it.red_off = reo;
    Batch b;
    std::memset(&b, 0, sizeof b);
    b.n_items = 1; b.one = it; b.total_blocks = blocks_for(F_EXT, d, it.ncols);
    set_bounds(p, b, (long long)ncols * d.G, false);
    k_extend<<<dim3((unsigned)b.total_blocks), 128, 0, st>>>(b, p->d_subs, p->d_tables, p->d_ws, 0);
    const long long n = (long long)it.ncols * d.G;
    k_basis_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(it, p->d_subs, p->d_tables, p->d_ws,
                                                              out + (long long)c * d.G);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- launchers
static inline dim3 grid1(int n) { return dim3((unsigned)n, 1, 1); }
static constexpr int FFT_SMEM = FFT_POINTS * 16;  // the most dynamic shared memory an FFT block may take

// Dynamic shared memory above 48 KiB must be opted into per kernel on the current device.
cudaError_t set_kernel_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_inv_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_fwd_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM);
  if (e == cudaSuccess) e = set_adj_kernel_attributes();
  if (e == cudaSuccess) e = set_tc_kernel_attributes();
  // the sweep's staging buffers take 32 x 2.4 KiB per SM at full occupancy: prefer shared memory
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tri<false, false, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tri<true, false, 2>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tri<false, false, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_tri<true, false, 4>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t launch_project(mdp_plan *p, const Batch *fb, int out_kind, const double2 *xi_user, double2 *out,
                           double2 *out_rec, cudaStream_t st) {
  const bool basis = xi_user == nullptr;
  const SubDesc *ds = p->d_subs;
  const double *tab = p->d_tables;
  double *ws = p->d_ws;
  const dim3 b8(32, 8), btri(32, TRI_WARPS);
#define MDP_LAUNCH(fam, ...)                      \
  do {                                            \
    if (fb[fam].total_blocks > 0) {               \
      prof_begin(p, fam, st);                     \
      __VA_ARGS__;                                \
      prof_end(p, fam, st);                       \
    }                                             \
  } while (0)
  if (basis) MDP_LAUNCH(F_EXT, k_extend<<<grid1(fb[F_EXT].total_blocks), 128, 0, st>>>(fb[F_EXT], ds, tab, ws, 0));
  if (basis) MDP_LAUNCH(F_RES, k_residual<false, false><<<grid1(fb[F_RES].total_blocks), b8, 0, st>>>(fb[F_RES], ds, tab, ws, xi_user));
  else MDP_LAUNCH(F_RES, k_residual<true, false><<<grid1(fb[F_RES].total_blocks), b8, 0, st>>>(fb[F_RES], ds, tab, ws, xi_user));
  if (basis) MDP_LAUNCH(F_FROWS, k_fwd_rows<false><<<grid1(fb[F_FROWS].total_blocks), b8, p->fft_smem, st>>>(fb[F_FROWS], ds, tab, ws));
  else MDP_LAUNCH(F_FROWS, k_fwd_rows<true><<<grid1(fb[F_FROWS].total_blocks), b8, p->fft_smem, st>>>(fb[F_FROWS], ds, tab, ws));
  if (p->tri_stages == 4) {
    if (basis) MDP_LAUNCH(F_TRI, k_tri<false, false, 4><<<grid1(fb[F_TRI].total_blocks), btri, tri_smem_bytes<false, 4>(), st>>>(fb[F_TRI], ds, tab, p->d_piv, ws));
    else MDP_LAUNCH(F_TRI, k_tri<true, false, 4><<<grid1(fb[F_TRI].total_blocks), btri, tri_smem_bytes<true, 4>(), st>>>(fb[F_TRI], ds, tab, p->d_piv, ws));
  } else {
    if (basis) MDP_LAUNCH(F_TRI, k_tri<false, false, 2><<<grid1(fb[F_TRI].total_blocks), btri, tri_smem_bytes<false, 2>(), st>>>(fb[F_TRI], ds, tab, p->d_piv, ws));
    else MDP_LAUNCH(F_TRI, k_tri<true, false, 2><<<grid1(fb[F_TRI].total_blocks), btri, tri_smem_bytes<true, 2>(), st>>>(fb[F_TRI], ds, tab, p->d_piv, ws));
  }
  if (basis) {
    MDP_LAUNCH(F_IROWS, k_inv_rows<false><<<grid1(fb[F_IROWS].total_blocks), b8, p->fft_smem, st>>>(fb[F_IROWS], ds, tab, ws, xi_user, out, out_kind));
    MDP_LAUNCH(F_ICOLS, k_inv_cols<false><<<grid1(fb[F_ICOLS].total_blocks), b8, 0, st>>>(fb[F_ICOLS], ds, tab, ws, xi_user, out, out_kind));
  } else {
    MDP_LAUNCH(F_IROWS, k_inv_rows<true><<<grid1(fb[F_IROWS].total_blocks), b8, p->fft_smem, st>>>(fb[F_IROWS], ds, tab, ws, xi_user, out, out_kind));
    MDP_LAUNCH(F_ICOLS, k_inv_cols<true><<<grid1(fb[F_ICOLS].total_blocks), b8, 0, st>>>(fb[F_ICOLS], ds, tab, ws, xi_user, out, out_kind));
  }
  if (fb[F_TCOLS].total_blocks > 0)
    MDP_LAUNCH(F_TCOLS, launch_inv_cols_tc(fb[F_TCOLS], ds, tab, ws, xi_user, out, out_kind, p->d_status, p->n_sm, st));
  if (out_rec)
    MDP_LAUNCH(F_IREC, k_inv_rec<<<grid1(fb[F_IREC].total_blocks), b8, 0, st>>>(fb[F_IREC], ds, tab, ws, out_rec, basis ? 0 : 1));
  return cudaGetLastError();
}

cudaError_t launch_adjoint(mdp_plan *p, const Batch *fb, int out_kind, const double2 *xi_user, const double2 *cot,
                           const double2 *cot_rec, double2 *grad_xi, double *grad_k, cudaStream_t st) {
  const bool basis = xi_user == nullptr;
  const SubDesc *ds = p->d_subs;
  const double *tab = p->d_tables;
  double *ws = p->d_ws;
  const dim3 b8(32, 8), btri(32, TRI_WARPS);
  if (grad_k) {  // forward recompute with every mode-space row kept, and the k-derivative sources
    if (basis) MDP_LAUNCH(F_EXT, k_extend<<<grid1(fb[F_EXT].total_blocks), 128, 0, st>>>(fb[F_EXT], ds, tab, ws, 1));
    if (basis) MDP_LAUNCH(F_RES, k_residual<false, true><<<grid1(fb[F_RES].total_blocks), b8, 0, st>>>(fb[F_RES], ds, tab, ws, xi_user));
    else MDP_LAUNCH(F_RES, k_residual<true, true><<<grid1(fb[F_RES].total_blocks), b8, 0, st>>>(fb[F_RES], ds, tab, ws, xi_user));
    if (basis) MDP_LAUNCH(F_FROWS, k_fwd_rows<false><<<grid1(fb[F_FROWS].total_blocks), b8, p->fft_smem, st>>>(fb[F_FROWS], ds, tab, ws));
    else MDP_LAUNCH(F_FROWS, k_fwd_rows<true><<<grid1(fb[F_FROWS].total_blocks), b8, p->fft_smem, st>>>(fb[F_FROWS], ds, tab, ws));
    if (basis) MDP_LAUNCH(F_TRI, k_tri<false, true, 2><<<grid1(fb[F_TRI].total_blocks), btri, TRI_WARPS * 2 * full_stage_bytes<false>(), st>>>(fb[F_TRI], ds, tab, p->d_piv, ws));
    else MDP_LAUNCH(F_TRI, k_tri<true, true, 2><<<grid1(fb[F_TRI].total_blocks), btri, TRI_WARPS * 2 * full_stage_bytes<true>(), st>>>(fb[F_TRI], ds, tab, p->d_piv, ws));
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_adjoint_tail(p, fb, out_kind, xi_user, cot, cot_rec, grad_xi, grad_k, st);
}

}  // namespace mdp
