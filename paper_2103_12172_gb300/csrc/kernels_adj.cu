// Adjoint of the projection columns and the wavenumber gradient (CUDA, sm_103a, FP64).
//
// For out_c = (P_gamma - I) xi_c = -Tr G^(h) R L^(h) W xi_c (Sections 3.2.2, 3.2.5) and a real
// loss with cotangent c = dLoss/d conj(out):
//   grad_xi_c = -W^T L^T R^T G^H Tr^T c_c   (+ c_c for P_gamma),
//   dLoss/dk  = Re sum_c [ <mu_c, A' u_c> - <R^T mu_c, s_c> ]   (+ Re <c_c, dxi_c/dk>, P kind),
// with mu_c = A^{-H} Tr^T c_c, u_c = G^(h) r_c, A' = dA/dk, s_c = (L' w_c + L w'_c)|_{M+}.
// Along x the sine transform S (unnormalised) diagonalises A: with yhat = S Tr^T c,
//   muhat_q = T_q^{-H} yhat_q,  mu = (2/Nx) S muhat,  <mu, A'u> = (2/Nx) sum_q <muhat_q, T_q' uhat_q>,
// so the adjoint is the forward path with gamma and the ring exchanging roles and the
// conjugate-transposed mode solve. Partial sums of the gradient are reduced per block in a
// fixed order and then per subdomain in item order (deterministic).
#include "kernels_common.cuh"

namespace mdp {

static inline dim3 g1(int n) { return dim3((unsigned)n, 1, 1); }
static constexpr int FFT_SMEM_ADJ = FFT_POINTS * 16;  // bytes of dynamic shared memory of the FFT kernels


// yhat(q, row) = sum_m c(m) sin(pi q m / Nx) of the 4 full gamma rows of the cotangent (and
// the receiver row): by FFT where the plan allows it (Nx a power of 2), else a direct sum.
//
// FFT form: a DST-I by one complex FFT of length Nx (dst1_post). One block: one row and fpb
// columns.
__device__ __forceinline__ void adj_rows_fft(const Item &it, const SubDesc &d, const double *tab, double *ws,
                                             const double2 *cot, const double2 *cot_rec, int local, double2 *sm) {
  __shared__ double2 tot[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int rr = local % 5, cblk = local / 5;
  if (rr == 4 && !(cot_rec && d.nrec >= 0)) return;   // uniform over the block
  const int b0 = cblk * d.fpb, nf = min(d.fpb, it.ncols - b0);
  const int N = d.Nx, H = N / 2;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  const double *sn = tab + d.sin_off;
  const int W = d.Px + 2, M4 = 4 * (d.Py - 2);
  // the row's values c(m) for m in [m0, m0 + cnt), column f at src(f) + (m - m0)
  const int m0 = rr == 4 ? d.mlo + 1 : d.mlo - 1, cnt = rr == 4 ? d.Px - 2 : W;
  const int g0 = rr == 0 ? 0 : rr == 1 ? W : rr == 2 ? 2 * W + M4 : 3 * W + M4;
  auto src = [&](int f) -> const double2 * {
    return rr == 4 ? cot_rec + d.rec_off + (long long)(it.col0 + b0 + f) * (d.Px - 2)
                   : cot + it.io_off + (long long)(b0 + f) * d.G + g0;
  };
  auto cv = [&](int f, int m) -> cplx {
    if (m < m0 || m >= m0 + cnt) return cmk(0.0, 0.0);
    const double2 v = src(f)[m - m0];
    return cmk(v.x, v.y);
  };
  // the twisted sequence, bit-reversed, for the pairs (m, N - m)
  for (int idx = tid; idx < d.fpb * (H + 1); idx += nt) {
    const int f = idx / (H + 1), j = idx - f * (H + 1);
    double2 *S = sm + (long long)f * N;
    if (j == 0) { S[0] = make_double2(0.0, 0.0); continue; }
    cplx xa = cmk(0.0, 0.0), xb = cmk(0.0, 0.0);
    if (f < nf) {
      xa = cv(f, j);
      if (2 * j != N) xb = cv(f, N - j);
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
  double *gr = ws + it.gr_off;
  for (int idx = tid; idx < nf * d.Nq; idx += nt) {
    const int f = idx % nf, q = idx / nf + 1;
    const double2 V = F[(long long)f * N + q];
    st2(gr + 2 * (((long long)rr * d.Nq + (q - 1)) * it.ncols + b0 + f), cmk(V.x, V.y));
  }
}

__global__ void __launch_bounds__(256) k_adj_rows(Batch bt, const SubDesc *subs, const double *tab, double *ws,
                                                  const double2 *cot, const double2 *cot_rec) {
  extern __shared__ double2 fft_sm[];
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_AFWD);
  const SubDesc &d = subs[it.sub];
  if (d.rows_fft) { adj_rows_fft(it, d, tab, ws, cot, cot_rec, local, fft_sm); return; }
  // direct: mode pair (q, Nx - q) per thread
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int q = (local / cb) * 8 + threadIdx.y + 1;
  if (b >= it.ncols || q > d.Nx / 2) return;
  const double *S = tab + d.sin_off;
  const int N2 = 2 * d.Nx, W = d.Px + 2, M4 = 4 * (d.Py - 2);
  const double2 *ct = cot + it.io_off + (long long)b * d.G;
  double *gr = ws + it.gr_off;
  const int q2 = d.Nx - q;
  for (int rr = 0; rr < 4; ++rr) {
    const int g0 = rr == 0 ? 0 : rr == 1 ? W : rr == 2 ? 2 * W + M4 : 3 * W + M4;
    cplx ao = cmk(0.0, 0.0), ae = cmk(0.0, 0.0);
    int j = (int)(((long long)q * (d.mlo - 1)) % N2);
    for (int mm = 0; mm < W; ++mm) {
      const int m = d.mlo - 1 + mm;
      const double2 cv = ct[g0 + mm];
      const cplx v = cmk(cv.x, cv.y);
      if (m & 1) ao = caxpy(S[j], v, ao); else ae = caxpy(S[j], v, ae);
      j += q;
      if (j >= N2) j -= N2;
    }
    st2(gr + 2 * (((long long)rr * d.Nq + (q - 1)) * it.ncols + b), cadd(ao, ae));
    if (q2 != q) st2(gr + 2 * (((long long)rr * d.Nq + (q2 - 1)) * it.ncols + b), csub(ao, ae));
  }
  if (cot_rec && d.nrec >= 0) {  // fifth row: the receiver cotangent at row nrec, m = mlo+1 .. mhi-1
    const double2 *cr = cot_rec + d.rec_off + (long long)(it.col0 + b) * (d.Px - 2);
    cplx ao = cmk(0.0, 0.0), ae = cmk(0.0, 0.0);
    int j = (int)(((long long)q * (d.mlo + 1)) % N2);
    for (int mm = 0; mm < d.Px - 2; ++mm) {
      const int m = d.mlo + 1 + mm;
      const cplx v = cmk(cr[mm].x, cr[mm].y);
      if (m & 1) ao = caxpy(S[j], v, ao); else ae = caxpy(S[j], v, ae);
      j += q;
      if (j >= N2) j -= N2;
    }
    st2(gr + 2 * ((4LL * d.Nq + (q - 1)) * it.ncols + b), cadd(ao, ae));
    if (q2 != q) st2(gr + 2 * ((4LL * d.Nq + (q2 - 1)) * it.ncols + b), csub(ao, ae));
  }
}

// The cotangent at the 4 gamma columns (mlo-1, mlo, mhi, mhi+1) of the middle rows nlo+1 ..
// nhi-1, gathered column-fastest into the r buffer ([4 (n - nlo - 1) + s][b], complex; r is free
// between the forward recompute and k_adj_ring_rows) for the sine transform in k_adj_tri. On an
// x-symmetric subdomain (mhi + 1 = Nx - (mlo - 1), mhi = Nx - mlo, so sin(pi q m'/Nx) =
// (-1)^(q+1) sin(pi q m/Nx) for the mirrored column m') the slots hold the pairs
// (c0 + c3, c0 - c3, c1 + c2, c1 - c2), and a mode needs two of them.
__global__ void __launch_bounds__(256) k_adj_cols(Batch bt, const SubDesc *subs, double *ws, const double2 *cot) {
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_ACOLS);
  const SubDesc &d = subs[it.sub];
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int t = (local / cb) * 8 + threadIdx.y;
  if (d.tc_cols && local == 0 && threadIdx.y == 0) {
    // the adjoint field's per-column exponents, maxed by k_adj_tri, start at 0
    int base[5];
    red_slots(d, it.ncols, base);
    int *ex = reinterpret_cast<int *>(ws + it.red_off + base[4] + 1);
    for (int i = threadIdx.x; i < it.ncols; i += 32) ex[i] = 0;
  }
  if (b >= it.ncols || t >= d.Py - 2) return;
  const double2 *c = cot + it.io_off + (long long)b * d.G + 2 * (d.Px + 2) + 4 * t;
  const cplx c0 = cmk(c[0].x, c[0].y), c1 = cmk(c[1].x, c[1].y), c2 = cmk(c[2].x, c[2].y), c3 = cmk(c[3].x, c[3].y);
  cplx v[4] = {c0, c1, c2, c3};
  if (d.xsym) {
    v[0] = cadd(c0, c3); v[1] = csub(c0, c3);
    v[2] = cadd(c1, c2); v[3] = csub(c1, c2);
  }
  double *r = ws + it.r_off;
#pragma unroll
  for (int s = 0; s < 4; ++s) st2(r + 2 * ((4LL * t + s) * it.ncols + b), v[s]);
}

// muhat = T_q^{-H} yhat for one (mode, column): U^H forward substitution (rows below the
// gamma band carry zero), then the transposed eliminations and row swaps from the top down to
// row 0. With DK the term Re <muhat, T_q' uhat> is accumulated as rows become final; muhat is
// kept on the ring rows nlo..nhi (a buffer, rows in matrix numbering).
// Operands are staged in shared memory by cp.async two rows ahead (sw: the warp's area; the
// active lanes are 0 .. nact-1): in the forward substitution a ring of 4 factor rows with the
// words holding their swap flags (row i reads rows i-1 and i-2 too) and 2 stages of right-hand
// side values; in the back sweep 2 stages of the factor row, the flag word, the stored z~ and
// the forward field uhat.
constexpr int ADJ_FR = 80;                      // factor row (<= 64 B) + flag word, per ring slot
constexpr int ADJ_RV = 5 * 32 * 16;             // right-hand side values [slot][lane], or the back stage
__host__ __device__ constexpr int adj_warp_smem() { return 4 * ADJ_FR + 2 * ADJ_RV; }

template <bool CF, bool DK>
__device__ __forceinline__ double adj_tri_body(const Item &it, const SubDesc &d, const double *tab,
                                               const uint8_t *pivtab, double *ws, bool rec, int b, int q, char *sw,
                                               int lane, int nact, unsigned mask) {
  constexpr int FW = CF ? 8 : 4;
  const int Nt = d.Nt, i0 = d.i0, nfirst = d.nfirst, nlo = d.nlo, nhi = d.nhi, Nq = d.Nq, nrec = d.nrec;
  const bool xsym = d.xsym;
  const double *F = tab + d.fact_off + (long long)(q - 1) * Nt * FW;
  const uint8_t *pv = pivtab + d.piv_off + (long long)(q - 1) * Nt;
  const int N2 = 2 * d.Nx;
  const double *S = tab + d.sin_off;
  const double sg0 = S[(q * (d.mlo - 1)) % N2], sg1 = S[(q * d.mlo) % N2];
  const double sg2 = S[(q * d.mhi) % N2], sg3 = S[(q * (d.mhi + 1)) % N2];
  const int nc = it.ncols;
  const double *gr = ws + it.gr_off;
  double *a = ws + it.a_off;
  const long long abase = (long long)(q - 1) * Nt * nc + b;
  auto aptr = [&](int i) { return a + 2 * (abase + (long long)i * nc); };
  // middle rows: the cotangent at the 4 gamma columns as gathered by k_adj_cols (column-fastest;
  // (sum, difference) pairs on x-symmetric subdomains: odd q takes the sums, even q the differences)
  const double *cc = ws + it.r_off;
  const int par = (q & 1) ? 0 : 1;
  char *fr_ring = sw, *rv = sw + 4 * ADJ_FR;
  // the factor row and the 4-byte word holding its swap flag (the flag table is 4-byte aligned
  // and padded to a multiple of 32 bytes, so the word never leaves it)
  auto fetch_row = [&](char *st, int i) {
    const double *src = F + (long long)i * FW;
    if (nact >= FW / 2) {
      if (lane < FW / 2) cp_async16(st + 16 * lane, src + 2 * lane);
    } else {
      for (int c = lane; c < FW / 2; c += nact) cp_async16(st + 16 * c, src + 2 * c);
    }
    if (lane == 0) {
      const uintptr_t ad = reinterpret_cast<uintptr_t>(pv + i);
      cp_async4(st + 64, reinterpret_cast<const void *>(ad & ~(uintptr_t)3));
    }
  };
  auto flag = [&](const char *st, int i) -> bool {
    const unsigned w = *reinterpret_cast<const unsigned *>(st + 64);
    return ((w >> (8 * (reinterpret_cast<uintptr_t>(pv + i) & 3))) & 0xffu) != 0;
  };
  // factor entry w (complex) of a staged row
  auto flc = [&](const char *st, int w) -> cplx {
    const double *r = reinterpret_cast<const double *>(st);
    return CF ? ld2(r + 2 * w) : cmk(r[w], 0.0);
  };
  auto flr = [&](const char *st, int w) -> double { return reinterpret_cast<const double *>(st)[CF ? 2 * w : w]; };
  // ---- forward substitution staging: factor row i, and the right-hand side of grid row i + nfirst
  auto fetch_fwd = [&](int i) {
    fetch_row(fr_ring + (i & 3) * ADJ_FR, i);
    const int n = i + nfirst;
    if (n >= nlo - 1 && n <= nhi + 1) {
      char *st = rv + (i & 1) * ADJ_RV + 16 * lane;
      const int rr = n == nlo - 1 ? 0 : n == nlo ? 1 : n == nhi ? 2 : n == nhi + 1 ? 3 : -1;
      if (rr >= 0) {
        cp_async16(st, gr + 2 * (((long long)rr * Nq + (q - 1)) * nc + b));
      } else {
        const long long s0 = 4LL * (n - nlo - 1);
        if (xsym) {
          cp_async16(st, cc + 2 * ((s0 + par) * nc + b));
          cp_async16(st + 512, cc + 2 * ((s0 + 2 + par) * nc + b));
        } else {
          for (int s_ = 0; s_ < 4; ++s_) cp_async16(st + 512 * s_, cc + 2 * ((s0 + s_) * nc + b));
        }
        if (rec && n == nrec) cp_async16(st + 4 * 512, gr + 2 * ((4LL * Nq + (q - 1)) * nc + b));
      }
    }
    cp_async_commit();
  };
  auto rhs = [&](int i) -> cplx {
    const int n = i + nfirst;
    if (n < nlo - 1 || n > nhi + 1) return cmk(0.0, 0.0);
    const double *st = reinterpret_cast<const double *>(rv + (i & 1) * ADJ_RV + 16 * lane);
    const bool dense = n == nlo - 1 || n == nlo || n == nhi || n == nhi + 1;
    if (dense) return ld2(st);
    cplx v = (rec && n == nrec) ? ld2(st + 4 * 64) : cmk(0.0, 0.0);
    if (xsym) {
      v = caxpy(sg0, ld2(st), v);
      v = caxpy(sg1, ld2(st + 64), v);
    } else {
      v = caxpy(sg0, ld2(st), v);
      v = caxpy(sg1, ld2(st + 64), v);
      v = caxpy(sg2, ld2(st + 128), v);
      v = caxpy(sg3, ld2(st + 192), v);
    }
    return v;
  };
  // Factor rows [rlo, rhi) of a complex mode are exactly real (plan: factor_mode); there the
  // products with the factors are real x complex.
  int rlo = 0, rhi = Nt;
  if (CF) {
    const double *sgm = tab + d.seg_off + 5 * (q - 1);
    rlo = (int)sgm[0];
    rhi = (int)sgm[1];
  }
  auto begin = [&]() { cp_async_wait<1>(); __syncwarp(mask); };
  auto end_fwd = [&](int i) {
    __syncwarp(mask);
    if (i + 2 < Nt) fetch_fwd(i + 2); else cp_async_commit();
  };
  for (int j = 0; j < 2; ++j) {
    if (i0 + j < Nt) fetch_fwd(i0 + j); else cp_async_commit();
  }
  // U^H zt = yhat, zt_i = conj(d_i) z_i, from the first nonzero row (i0) up
  cplx t1 = cmk(0.0, 0.0), t2 = cmk(0.0, 0.0);
  auto fstep_c = [&](int i) {
    begin();
    const char *r0 = fr_ring + (i & 3) * ADJ_FR, *r1 = fr_ring + ((i - 1) & 3) * ADJ_FR, *r2 = fr_ring + ((i - 2) & 3) * ADJ_FR;
    cplx v = rhs(i);
    if (i - 1 >= i0) v = cfms(v, cconj(flc(r1, 2)), t1);
    if (i - 2 >= i0 && flag(r2, i - 2)) v = cfms(v, cconj(flc(r2, 3)), t2);
    const cplx z = cmul(cconj(flc(r0, 1)), v);
    end_fwd(i);
    st2(aptr(i), z);
    t2 = t1; t1 = v;
  };
  auto fstep_r = [&](int i) {   // rows i-2, i-1, i real
    begin();
    const char *r0 = fr_ring + (i & 3) * ADJ_FR, *r1 = fr_ring + ((i - 1) & 3) * ADJ_FR, *r2 = fr_ring + ((i - 2) & 3) * ADJ_FR;
    cplx v = rhs(i);
    if (i - 1 >= i0) v = caxpy(-flr(r1, 2), t1, v);
    if (i - 2 >= i0 && flag(r2, i - 2)) v = caxpy(-flr(r2, 3), t2, v);
    const double di = flr(r0, 1);
    end_fwd(i);
    st2(aptr(i), cmk(di * v.re, di * v.im));
    t2 = t1; t1 = v;
  };
  {
    int i = i0;
    if (CF) for (const int e = min(max(rlo + 2, i), Nt); i < e; ++i) fstep_c(i);
    for (const int e = CF ? max(rhi, i) : Nt; i < e; ++i) fstep_r(i);
    for (; i < Nt; ++i) fstep_c(i);
  }
  // the stored z~ are read back below by this thread's asynchronous copies: order them after
  // its stores
  __threadfence_block();
  // z = P_0 E_0^H ... P_{N-2} E_{N-2}^H z; position i+1 is final after step i
  const double *dT = tab + d.dT_off + (long long)(q - 1) * Nt * 6;
  const double *y = ws + it.y_off;
  const long long ybase = (long long)(q - 1) * Nt * nc + b;
  // ---- back sweep staging (rows Nt-2 .. 0): factor row, flag word, z~ (rows >= i0) and, with
  // DK, uhat of the same row
  auto bst = [&](int i) -> char * { return rv + (i & 1) * ADJ_RV; };
  auto fetch_back = [&](int i) {
    char *st = bst(i);
    fetch_row(st, i);
    if (i >= i0) cp_async16(st + 80 + 16 * lane, aptr(i));
    if (DK) cp_async16(st + 80 + 512 + 16 * lane, y + 2 * (ybase + (long long)i * nc));
    cp_async_commit();
  };
  auto end_back = [&](int i) {
    __syncwarp(mask);
    if (i - 2 >= 0) fetch_back(i - 2); else cp_async_commit();
  };
  // Re <muhat, T_q' uhat>: T_q' is (da, ddk, da) with real constants on rows 1 .. Nt-2 (the
  // k-derivatives of the interior coefficients), so those rows accumulate
  // s_off = sum Re conj(mu_j)(u_{j-1} + u_{j+1}) and s_dg = sum Re conj(mu_j) u_j; the two end
  // rows (Sommerfeld or Dirichlet) take their tabulated entries.
  double dk = 0.0, s_off = 0.0, s_dg = 0.0;
  cplx uj1 = cmk(0.0, 0.0), uj = DK ? ld2(y + 2 * (ybase + (long long)(Nt - 1) * nc)) : cmk(0.0, 0.0);
  const int jlo = nlo - nfirst, jhi = nhi - nfirst;
  int emax = 0;   // largest biased exponent of muhat on the inner middle rows (integer compares only)
  auto bexp = [](double v) { return (__double2hiint(v) >> 20) & 0x7ff; };
  // ujm: uhat(j - 1)
  auto emit = [&](int j, cplx mu, cplx ujm) {
    if (DK) {
      if (j == 0 || j == Nt - 1) {
        const double *t = dT + 6 * j;
        cplx v = cmul(ld2(t), ujm);
        v = cadd(v, cmul(ld2(t + 2), uj));
        v = cadd(v, cmul(ld2(t + 4), uj1));
        dk = fma(mu.re, v.re, fma(mu.im, v.im, dk));
      } else {
        s_off = fma(mu.re, ujm.re + uj1.re, fma(mu.im, ujm.im + uj1.im, s_off));
        s_dg = fma(mu.re, uj.re, fma(mu.im, uj.im, s_dg));
      }
      uj1 = uj; uj = ujm;
    }
    if (j >= jlo && j <= jhi) st2(aptr(j), mu);
    if (j >= jlo + 2 && j <= jhi - 2) emax = max(emax, max(bexp(mu.re), bexp(mu.im)));   // the rows the ring columns sum
  };
  cplx up = ld2(aptr(Nt - 1));
  for (int j = 0; j < 2; ++j) {
    if (Nt - 2 - j >= 0) fetch_back(Nt - 2 - j); else cp_async_commit();
  }
  auto bstep = [&](int i, bool complex_row) {
    begin();
    const char *st = bst(i);
    const cplx zi0 = i >= i0 ? ld2(reinterpret_cast<const double *>(st + 80 + 16 * lane)) : cmk(0.0, 0.0);
    const cplx ujm = DK ? ld2(reinterpret_cast<const double *>(st + 80 + 512 + 16 * lane)) : cmk(0.0, 0.0);
    const cplx zi = complex_row ? cfms(zi0, cconj(flc(st, 0)), up) : caxpy(-flr(st, 0), up, zi0);
    const bool swp = flag(st, i);
    end_back(i);
    if (swp) emit(i + 1, zi, ujm);
    else { emit(i + 1, up, ujm); up = zi; }
  };
  {
    int i = Nt - 2;
    if (CF) for (; i >= rhi; --i) bstep(i, true);
    for (const int e = CF ? rlo : 0; i >= e; --i) bstep(i, false);
    for (; i >= 0; --i) bstep(i, true);
  }
  emit(0, up, cmk(0.0, 0.0));
  if (DK && Nt >= 3) dk = fma(dT[6 + 0], s_off, fma(dT[6 + 2], s_dg, dk));
  if (d.tc_cols) {   // per column, over every mode: the common scale of the tensor-core ring sums
    int base[5];
    red_slots(d, nc, base);
    atomicMax(reinterpret_cast<int *>(ws + it.red_off + base[4] + 1) + b, emax);
  }
  return dk;
}

template <bool DK>
__global__ void __launch_bounds__(128, 7) k_adj_tri(Batch bt, const SubDesc *subs, const double *tab, const uint8_t *pivtab,
                                                 double *ws, int has_rec) {
  __shared__ double sh[128];
  extern __shared__ __align__(16) char adj_sm[];
  Item it; int local;
  locate(bt, bt.order ? bt.order[blockIdx.x] : (int)blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_ATRI);
  const SubDesc &d = subs[it.sub];
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int q = (local / cb) * 4 + threadIdx.y + 1;
  const bool act = b < it.ncols && q <= d.Nq;
  const unsigned mask = __ballot_sync(0xffffffffu, act);   // a warp shares q; its active lanes are 0 .. nact-1
  double dk = 0.0;
  if (act) {
    char *sw = adj_sm + threadIdx.y * adj_warp_smem();
    dk = d.cplx ? adj_tri_body<true, DK>(it, d, tab, pivtab, ws, has_rec && d.nrec >= 0, b, q, sw, threadIdx.x,
                                         __popc(mask), mask)
                : adj_tri_body<false, DK>(it, d, tab, pivtab, ws, has_rec && d.nrec >= 0, b, q, sw, threadIdx.x,
                                          __popc(mask), mask);
  }
  if (DK) {
    const double s = block_sum<128>(dk * (2.0 / d.Nx), sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) ws[it.red_off + local] = s;   // slot base 0: k_adj_tri
  }
}

// mu on the 4 full ring rows (into the r buffer, complex [R][b]); DK: -Re <mu, s>.
// FFT form (as for the forward path's gamma rows): mu(m) = (2/Nx) F_m with F the DST-I of
// muhat (dst1_post). One block: one ring row and fpb columns.
template <bool DK>
__device__ __forceinline__ double adj_ring_rows_fft(const Item &it, const SubDesc &d, const double *tab, double *ws,
                                                    int local, double2 *sm) {
  __shared__ double2 tot[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int rr = local & 3, cblk = local >> 2;
  const int b0 = cblk * d.fpb, nf = min(d.fpb, it.ncols - b0);
  const int N = d.Nx, H = N / 2;
  int lg = 0;
  while ((1 << lg) < N) ++lg;
  const double *sn = tab + d.sin_off;
  const int P = d.Px, Mr = 4 * (d.Py - 4);
  const int n = rr == 0 ? d.nlo : rr == 1 ? d.nlo + 1 : rr == 2 ? d.nhi - 1 : d.nhi;
  const int j = n - d.nfirst;
  const double *a = ws + it.a_off;
  const long long qstride = (long long)d.Nt * it.ncols;
  auto mv = [&](int q, int f) -> cplx {   // muhat(q) of column b0 + f, q = 1 .. N-1
    return ld2(a + 2 * ((long long)(q - 1) * qstride + (long long)j * it.ncols + b0 + f));
  };
  // the twisted sequence, bit-reversed, for the pairs (q, N - q); the column is fastest
  for (int idx = tid; idx < d.fpb * (H + 1); idx += nt) {
    const int f = idx % d.fpb, q = idx / d.fpb;
    double2 *S = sm + (long long)f * N;
    if (q == 0) { S[0] = make_double2(0.0, 0.0); continue; }
    cplx xa = cmk(0.0, 0.0), xb = cmk(0.0, 0.0);
    if (f < nf) {
      xa = mv(q, f);
      if (2 * q != N) xb = mv(N - q, f);
    }
    if (2 * q == N) { S[brev_lg(q, lg)] = make_double2(2.0 * xa.re, 2.0 * xa.im); continue; }
    cplx ya, yb;
    dst1_twist(xa, xb, sn[q], ya, yb);
    S[brev_lg(q, lg)] = make_double2(ya.re, ya.im);
    S[brev_lg(N - q, lg)] = make_double2(yb.re, yb.im);
  }
  __syncthreads();
  fft_r2_stages(sm, d.fpb, N, lg, sn);
  double2 *F = sm + (long long)d.fpb * N;
  dst1_post(sm, F, d.fpb, N, tot);
  const int rb = rr == 0 ? 0 : rr == 1 ? P : rr == 2 ? 2 * P + Mr : 3 * P + Mr;
  const double sc = 2.0 / N;
  double dk = 0.0;
  for (int idx = tid; idx < nf * P; idx += nt) {
    const int f = idx % nf, dm = idx / nf;
    const double2 V = F[(long long)f * N + d.mlo + dm];
    const cplx acc = cmk(sc * V.x, sc * V.y);
    const long long o = (long long)(rb + dm) * it.ncols + b0 + f;
    st2(ws + it.r_off + 2 * o, acc);
    if (DK) {
      const cplx s = ld2(ws + it.s_off + 2 * o);
      dk -= acc.re * s.re + acc.im * s.im;
    }
  }
  return dk;
}

template <bool DK>
__global__ void __launch_bounds__(256) k_adj_ring_rows(Batch bt, const SubDesc *subs, const double *tab, double *ws) {
  extern __shared__ double2 fft_sm[];
  __shared__ double sh[256];
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_ARING);
  const SubDesc &d = subs[it.sub];
  double dk = 0.0;
  if (d.rows_fft) {
    dk = adj_ring_rows_fft<DK>(it, d, tab, ws, local, fft_sm);
  } else {
    const int cb = (it.ncols + 31) >> 5;
    const int b = (local % cb) * 32 + threadIdx.x;
    const int task = (local / cb) * 8 + threadIdx.y;
    const int P = d.Px, Mr = 4 * (d.Py - 4);
    if (b < it.ncols && task < 4 * P) {
      const int rr = task / P, m = d.mlo + task % P;
      const int n = rr == 0 ? d.nlo : rr == 1 ? d.nlo + 1 : rr == 2 ? d.nhi - 1 : d.nhi;
      const int j = n - d.nfirst;
      const double *Si = tab + d.sin_off + 2 * d.Nx;
      const int N2 = 2 * d.Nx;
      const double *a = ws + it.a_off;
      const long long qstride = (long long)d.Nt * it.ncols;
      const long long base = (long long)j * it.ncols + b;
      cplx acc = cmk(0.0, 0.0);
      int jj = m % N2;
      for (int q = 1; q <= d.Nq; ++q) {
        acc = caxpy(Si[jj], ld2(a + 2 * (base + (long long)(q - 1) * qstride)), acc);
        jj += m;
        if (jj >= N2) jj -= N2;
      }
      const int rb = rr == 0 ? 0 : rr == 1 ? P : rr == 2 ? 2 * P + Mr : 3 * P + Mr;
      const long long o = (long long)(rb + m - d.mlo) * it.ncols + b;
      st2(ws + it.r_off + 2 * o, acc);
      if (DK) {
        const cplx s = ld2(ws + it.s_off + 2 * o);
        dk = -(acc.re * s.re + acc.im * s.im);
      }
    }
  }
  if (DK) {
    int base[5];
    red_slots(d, it.ncols, base);
    const double s = block_sum<256>(dk, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) ws[it.red_off + base[1] + local] = s;
  }
}

// mu on the ring's middle rows nlo+2 .. nhi-2 at the columns mlo, mlo+1, mhi-1, mhi
template <bool DK>
__global__ void __launch_bounds__(256) k_adj_ring_cols(Batch bt, const SubDesc *subs, const double *tab, double *ws) {
  __shared__ double sh[256];
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_ARINGC);
  const SubDesc &d = subs[it.sub];
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int t = (local / cb) * 8 + threadIdx.y;
  double dk = 0.0;
  if (b < it.ncols && t < d.Py - 4) {
    const int n = d.nlo + 2 + t, j = n - d.nfirst;
    const double *Si = tab + d.sin_off + 2 * d.Nx;
    const int N2 = 2 * d.Nx;
    const int ms[4] = {d.mlo, d.mlo + 1, d.mhi - 1, d.mhi};
    int jj[4] = {ms[0] % N2, ms[1] % N2, ms[2] % N2, ms[3] % N2};
    const double *a = ws + it.a_off;
    const long long qstride = (long long)d.Nt * it.ncols;
    const long long base = (long long)j * it.ncols + b;
    cplx acc[4] = {cmk(0, 0), cmk(0, 0), cmk(0, 0), cmk(0, 0)};
    if (d.xsym) {
      // mhi = Nx - mlo: sin(pi q (Nx - m)/Nx) = sin(pi q m/Nx) for odd q and its negative for
      // even q, so odd-q and even-q partial sums at mlo, mlo+1 give all four columns
      cplx e0 = cmk(0, 0), o0 = cmk(0, 0), e1 = cmk(0, 0), o1 = cmk(0, 0);
      int q = 1;
      for (; q + 1 <= d.Nq; q += 2) {
        const cplx va = ld2(a + 2 * (base + (long long)(q - 1) * qstride));
        const cplx vb = ld2(a + 2 * (base + (long long)q * qstride));
        e0 = caxpy(Si[jj[0]], va, e0); e1 = caxpy(Si[jj[1]], va, e1);
        jj[0] += ms[0]; if (jj[0] >= N2) jj[0] -= N2;
        jj[1] += ms[1]; if (jj[1] >= N2) jj[1] -= N2;
        o0 = caxpy(Si[jj[0]], vb, o0); o1 = caxpy(Si[jj[1]], vb, o1);
        jj[0] += ms[0]; if (jj[0] >= N2) jj[0] -= N2;
        jj[1] += ms[1]; if (jj[1] >= N2) jj[1] -= N2;
      }
      if (q <= d.Nq) {
        const cplx va = ld2(a + 2 * (base + (long long)(q - 1) * qstride));
        e0 = caxpy(Si[jj[0]], va, e0); e1 = caxpy(Si[jj[1]], va, e1);
      }
      acc[0] = cadd(e0, o0); acc[3] = csub(e0, o0);
      acc[1] = cadd(e1, o1); acc[2] = csub(e1, o1);
    } else {
      for (int q = 1; q <= d.Nq; ++q) {
        const cplx v = ld2(a + 2 * (base + (long long)(q - 1) * qstride));
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          acc[s] = caxpy(Si[jj[s]], v, acc[s]);
          jj[s] += ms[s];
          if (jj[s] >= N2) jj[s] -= N2;
        }
      }
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const long long o = (long long)(2 * d.Px + 4 * t + s) * it.ncols + b;
      st2(ws + it.r_off + 2 * o, acc[s]);
      if (DK) {
        const cplx sv = ld2(ws + it.s_off + 2 * o);
        dk -= acc[s].re * sv.re + acc[s].im * sv.im;
      }
    }
  }
  if (DK) {
    int base[5];
    red_slots(d, it.ncols, base);
    const double s = block_sum<256>(dk, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) ws[it.red_off + base[2] + local] = s;
  }
}

// grad_xi = -(L mu|ring) on gamma (+ cot for P_gamma); DK with basis densities and the P kind:
// + Re <cot, dxi/dk>
template <bool CIN, bool DK>
__global__ void __launch_bounds__(256) k_adj_gamma(Batch bt, const SubDesc *subs, const double *tab, double *ws,
                                                   const double2 *cot, double2 *grad_xi, int kind) {
  __shared__ double sh[256];
  Item it; int local;
  locate(bt, blockIdx.x, it, local);
  MDP_CHECK_ITEM(bt, subs, it, local, F_AGAM);
  const SubDesc &d = subs[it.sub];
  const int cb = (it.ncols + 31) >> 5;
  const int b = (local % cb) * 32 + threadIdx.x;
  const int g = (local / cb) * 8 + threadIdx.y;
  double dk = 0.0;
  if (b < it.ncols && g < d.G) {
    int n, m;
    gamma_node(d, g, n, m);
    cplx acc = cmk(0.0, 0.0);
#pragma unroll
    for (int dn = -1; dn <= 1; ++dn) {
#pragma unroll
      for (int dm = -1; dm <= 1; ++dm) {
        const int ri = ring_index(d, n + dn, m + dm);
        if (ri < 0) continue;
        const int nb = (dn != 0) + (dm != 0);
        const double c = nb == 0 ? d.c0 : nb == 1 ? d.c1 : d.c2;
        acc = caxpy(c, ld2(ws + it.r_off + 2 * ((long long)ri * it.ncols + b)), acc);
      }
    }
    const long long io = it.io_off + (long long)b * d.G + g;
    cplx gx = cmk(-acc.re, -acc.im);
    if (kind == MDP_OUT_P) {
      const cplx c = cmk(cot[io].x, cot[io].y);
      gx = cadd(gx, c);
      if (DK && !CIN && (int)tab[d.geo_off + 4 * g] == col_side(d, it.col0 + b)) {
        const double dxi = ws[it.xi_off + (long long)d.G * it.ncols + (long long)g * it.ncols + b];
        dk = c.re * dxi;
      }
    }
    if (grad_xi) grad_xi[io] = make_double2(gx.re, gx.im);
  }
  if (DK) {
    int base[5];
    red_slots(d, it.ncols, base);
    const double s = block_sum<256>(dk, sh);
    if (threadIdx.x == 0 && threadIdx.y == 0) ws[it.red_off + base[3] + local] = s;
  }
}

// per item: the sum of its partials in slot order; then per subdomain in item order
__global__ void __launch_bounds__(256) k_red_items(const Item *items, const SubDesc *subs, double *ws) {
  __shared__ double sh[256];
  const Item it = items[blockIdx.x];
  const SubDesc &d = subs[it.sub];
  int base[5];
  red_slots(d, it.ncols, base);
  double v = 0.0;
  for (int i = threadIdx.x; i < base[4]; i += 256) v += ws[it.red_off + i];
  // block_sum expects a (32 x 8) layout; use a flat block of 256
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) ws[it.red_off + base[4]] = sh[0];
}

__global__ void k_red_subs(const Item *items, int n_items, const SubDesc *subs, const double *ws, double *grad_k) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = 0; i < n_items; ++i) {
    const Item it = items[i];
    int base[5];
    red_slots(subs[it.sub], it.ncols, base);
    grad_k[it.sub] += ws[it.red_off + base[4]];
  }
}

cudaError_t set_adj_kernel_attributes() {
  cudaError_t e = cudaFuncSetAttribute(k_adj_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM_ADJ);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_adj_ring_rows<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM_ADJ);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_adj_ring_rows<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, FFT_SMEM_ADJ);
  return e;
}

cudaError_t launch_adjoint_tail(mdp_plan *p, const Batch *fb, int out_kind, const double2 *xi_user, const double2 *cot,
                                const double2 *cot_rec, double2 *grad_xi, double *grad_k, cudaStream_t st) {
  const SubDesc *ds = p->d_subs;
  const double *tab = p->d_tables;
  double *ws = p->d_ws;
  const dim3 b8(32, 8), b4(32, 4);
  const bool dk = grad_k != nullptr, basis = xi_user == nullptr;
#define ADJ_LAUNCH(fam, ...)                      \
  do {                                            \
    if (fb[fam].total_blocks > 0) {               \
      prof_begin(p, fam, st);                     \
      __VA_ARGS__;                                \
      prof_end(p, fam, st);                       \
    }                                             \
  } while (0)
  ADJ_LAUNCH(F_AFWD, k_adj_rows<<<g1(fb[F_AFWD].total_blocks), b8, p->fft_smem, st>>>(fb[F_AFWD], ds, tab, ws, cot, cot_rec));
  ADJ_LAUNCH(F_ACOLS, k_adj_cols<<<g1(fb[F_ACOLS].total_blocks), b8, 0, st>>>(fb[F_ACOLS], ds, ws, cot));
  if (dk) ADJ_LAUNCH(F_ATRI, k_adj_tri<true><<<g1(fb[F_ATRI].total_blocks), b4, 4 * adj_warp_smem(), st>>>(fb[F_ATRI], ds, tab, p->d_piv, ws, cot_rec ? 1 : 0));
  else ADJ_LAUNCH(F_ATRI, k_adj_tri<false><<<g1(fb[F_ATRI].total_blocks), b4, 4 * adj_warp_smem(), st>>>(fb[F_ATRI], ds, tab, p->d_piv, ws, cot_rec ? 1 : 0));
  if (dk) {
    ADJ_LAUNCH(F_ARING, k_adj_ring_rows<true><<<g1(fb[F_ARING].total_blocks), b8, p->fft_smem, st>>>(fb[F_ARING], ds, tab, ws));
    ADJ_LAUNCH(F_ARINGC, k_adj_ring_cols<true><<<g1(fb[F_ARINGC].total_blocks), b8, 0, st>>>(fb[F_ARINGC], ds, tab, ws));
    ADJ_LAUNCH(F_ATCOLS, launch_adj_cols_tc(fb[F_ATCOLS], ds, tab, ws, true, p->d_status, p->n_sm, st));
  } else {
    ADJ_LAUNCH(F_ARING, k_adj_ring_rows<false><<<g1(fb[F_ARING].total_blocks), b8, p->fft_smem, st>>>(fb[F_ARING], ds, tab, ws));
    ADJ_LAUNCH(F_ARINGC, k_adj_ring_cols<false><<<g1(fb[F_ARINGC].total_blocks), b8, 0, st>>>(fb[F_ARINGC], ds, tab, ws));
    ADJ_LAUNCH(F_ATCOLS, launch_adj_cols_tc(fb[F_ATCOLS], ds, tab, ws, false, p->d_status, p->n_sm, st));
  }
  if (dk && basis)
    ADJ_LAUNCH(F_AGAM, k_adj_gamma<false, true><<<g1(fb[F_AGAM].total_blocks), b8, 0, st>>>(fb[F_AGAM], ds, tab, ws, cot, grad_xi, out_kind));
  else if (dk)
    ADJ_LAUNCH(F_AGAM, k_adj_gamma<true, true><<<g1(fb[F_AGAM].total_blocks), b8, 0, st>>>(fb[F_AGAM], ds, tab, ws, cot, grad_xi, out_kind));
  else if (grad_xi)
    ADJ_LAUNCH(F_AGAM, k_adj_gamma<true, false><<<g1(fb[F_AGAM].total_blocks), b8, 0, st>>>(fb[F_AGAM], ds, tab, ws, cot, grad_xi, out_kind));
  if (dk) {
    k_red_items<<<fb[F_ATRI].n_items, 256, 0, st>>>(fb[F_ATRI].items, ds, ws);
    k_red_subs<<<1, 32, 0, st>>>(fb[F_ATRI].items, fb[F_ATRI].n_items, ds, ws, grad_k);
  }
  return cudaGetLastError();
}

}  // namespace mdp
