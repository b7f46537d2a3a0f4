// Device helpers shared by the projection and adjoint kernels: complex FP64 arithmetic,
// batch addressing, and the index maps of gamma (the 2-node ring around M+) and of the ring
// that carries r = L^(h) w restricted to M+.
#pragma once
#include "mdp_internal.h"

namespace mdp {

// ---------------------------------------------------------------- complex helpers
struct cplx { double re, im; };
__device__ __forceinline__ cplx cmk(double a, double b) { return {a, b}; }
__device__ __forceinline__ cplx cadd(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
// a - b*c
__device__ __forceinline__ cplx cfms(cplx a, cplx b, cplx c) {
  return {fma(-b.re, c.re, fma(b.im, c.im, a.re)), fma(-b.re, c.im, fma(-b.im, c.re, a.im))};
}
// a + s*c (s real)
__device__ __forceinline__ cplx caxpy(double s, cplx c, cplx a) { return {fma(s, c.re, a.re), fma(s, c.im, a.im)}; }
__device__ __forceinline__ cplx ld2(const double *p) {
  double2 v = *reinterpret_cast<const double2 *>(p);
  return {v.x, v.y};
}
__device__ __forceinline__ void st2(double *p, cplx v) { *reinterpret_cast<double2 *>(p) = make_double2(v.re, v.im); }

// ---------------------------------------------------------------- asynchronous copies
// Asynchronous global -> shared copies (cp.async): operands of rows ahead are in flight while
// the current row is swept, without holding registers for them.
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------- batch addressing
__device__ __forceinline__ void locate(const Batch &b, int blk, Item &it, int &local) {
  if (b.items == nullptr) { it = b.one; local = blk; return; }
  int lo = 0, hi = b.n_items - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (b.prefix[mid] <= blk) lo = mid; else hi = mid - 1;
  }
  it = b.items[lo];
  local = blk - b.prefix[lo];
}

// ---------------------------------------------------------------- bounds checks (MDP_CHECKED)
// The first violation is recorded as MDP_ERR_BOUNDS in the status word; the access is skipped.
__device__ __forceinline__ void flag_bounds(int *status) {
  if (status) atomicCAS(status, 0, (int)MDP_ERR_BOUNDS);
}
// A block's item against the call's ranges: the subdomain index, the column range, the block
// number within the kernel family, every workspace slice of the item, every table of the
// subdomain, its pivot flags, and its columns of the output (or density, cotangent) array.
static __device__ __noinline__ bool item_in_bounds(const Batch &bt, const SubDesc *subs, const Item &it, int local, int fam,
                                            bool grad) {
  bool ok = it.sub >= 0 && it.sub < bt.n_subs && it.ncols >= 1 && local >= 0;
  if (ok) {
    const SubDesc &d = subs[it.sub];
    ok = it.col0 >= 0 && it.col0 + it.ncols <= d.n_cols && local < blocks_for(fam, d, it.ncols);
    long long xi, r, gr, y, a, s, red, tot;
    item_workspace(d, it.ncols, grad, xi, r, gr, y, a, s, red, tot);
    auto in_ws = [&](long long off, long long n) { return off >= 0 && off + n <= bt.ws_n; };
    ok = ok && in_ws(it.xi_off, r - xi) && in_ws(it.r_off, gr - r) && in_ws(it.gr_off, y - gr) &&
         in_ws(it.y_off, a - y) && in_ws(it.red_off, tot - red) &&
         (!grad || (in_ws(it.a_off, s - a) && in_ws(it.s_off, red - s)));
    auto in_tab = [&](long long off, long long n) { return off >= 0 && off + n <= bt.tab_n; };
    const long long qt = (long long)d.Nq * d.Nt;
    ok = ok && in_tab(d.fact_off, qt * (d.cplx ? 8 : 4)) && in_tab(d.dT_off, qt * 6) && in_tab(d.sin_off, 4LL * d.Nx) &&
         in_tab(d.geo_off, 4LL * d.G) && in_tab(d.seg_off, 5LL * d.Nq) && in_tab(d.fs_off, (long long)d.Nq * d.NYf * FSW) &&
         (!d.tc_cols || in_tab(d.tcb_off, 256LL * ((d.Nq + 15) / 16)));
    ok = ok && d.piv_off >= 0 && d.piv_off + qt <= bt.piv_n;
    ok = ok && it.io_off >= 0 && it.io_off + (long long)it.ncols * d.G <= bt.out_n;
  }
  if (!ok) flag_bounds(bt.status);
  return ok;
}
// kernels: leave the block (uniformly: the item is the block's) when its item fails the checks
#define MDP_CHECK_ITEM(bt, subs, it, local, fam)                                                \
  do {                                                                                          \
    if (MDP_CHECKED && !item_in_bounds(bt, subs, it, local, fam, bt.grad != 0)) return;         \
  } while (0)

// gamma index of node (n, m), or -1 (row-major order of the 2-node ring around M+)
__device__ __forceinline__ int gamma_index(const SubDesc &d, int n, int m) {
  if (n < d.nlo - 1 || n > d.nhi + 1 || m < d.mlo - 1 || m > d.mhi + 1) return -1;
  const int W = d.Px + 2, Mr = d.Py - 2;
  const int dm = m - (d.mlo - 1);
  if (n == d.nlo - 1) return dm;
  if (n == d.nlo) return W + dm;
  if (n == d.nhi) return 2 * W + 4 * Mr + dm;
  if (n == d.nhi + 1) return 3 * W + 4 * Mr + dm;
  int slot = (m == d.mlo - 1) ? 0 : (m == d.mlo) ? 1 : (m == d.mhi) ? 2 : (m == d.mhi + 1) ? 3 : -1;
  if (slot < 0) return -1;
  return 2 * W + 4 * (n - d.nlo - 1) + slot;
}

// node of ring index ri (row-major order of the 2-node ring inside M+)
__device__ __forceinline__ void ring_node(const SubDesc &d, int ri, int &n, int &m) {
  const int P = d.Px, Mr = 4 * (d.Py - 4);
  if (ri < P) { n = d.nlo; m = d.mlo + ri; return; }
  if (ri < 2 * P) { n = d.nlo + 1; m = d.mlo + ri - P; return; }
  if (ri < 2 * P + Mr) {
    const int t = ri - 2 * P, slot = t & 3;
    n = d.nlo + 2 + (t >> 2);
    m = slot == 0 ? d.mlo : slot == 1 ? d.mlo + 1 : slot == 2 ? d.mhi - 1 : d.mhi;
    return;
  }
  if (ri < 3 * P + Mr) { n = d.nhi - 1; m = d.mlo + ri - 2 * P - Mr; return; }
  n = d.nhi; m = d.mlo + ri - 3 * P - Mr;
}

// ring index of node (n, m), or -1
__device__ __forceinline__ int ring_index(const SubDesc &d, int n, int m) {
  if (n < d.nlo || n > d.nhi || m < d.mlo || m > d.mhi) return -1;
  const int P = d.Px, Mr = 4 * (d.Py - 4);
  if (n == d.nlo) return m - d.mlo;
  if (n == d.nlo + 1) return P + m - d.mlo;
  if (n == d.nhi - 1) return 2 * P + Mr + m - d.mlo;
  if (n == d.nhi) return 3 * P + Mr + m - d.mlo;
  const int slot = m == d.mlo ? 0 : m == d.mlo + 1 ? 1 : m == d.mhi - 1 ? 2 : m == d.mhi ? 3 : -1;
  if (slot < 0) return -1;
  return 2 * P + 4 * (n - d.nlo - 2) + slot;
}

// node of gamma index g
__device__ __forceinline__ void gamma_node(const SubDesc &d, int g, int &n, int &m) {
  const int W = d.Px + 2, M4 = 4 * (d.Py - 2);
  if (g < W) { n = d.nlo - 1; m = d.mlo - 1 + g; return; }
  if (g < 2 * W) { n = d.nlo; m = d.mlo - 1 + g - W; return; }
  if (g < 2 * W + M4) {
    const int t = g - 2 * W, slot = t & 3;
    n = d.nlo + 1 + (t >> 2);
    m = slot == 0 ? d.mlo - 1 : slot == 1 ? d.mlo : slot == 2 ? d.mhi : d.mhi + 1;
    return;
  }
  if (g < 3 * W + M4) { n = d.nhi; m = d.mlo - 1 + g - 2 * W - M4; return; }
  n = d.nhi + 1; m = d.mlo - 1 + g - 3 * W - M4;
}

__device__ __forceinline__ cplx cconj(cplx a) { return {a.re, -a.im}; }

// side (1..4) of basis column c
__device__ __forceinline__ int col_side(const SubDesc &d, int c) { return (c % (4 * d.n_modes)) / d.n_modes + 1; }

// density value xi(c, g) for the item's column b (basis: owner check; user: complex array)
template <bool CIN>
__device__ __forceinline__ cplx density(const SubDesc &d, const Item &it, const double *ws, const double *tab,
                                        const double2 *xi_user, int b, int g) {
  if (MDP_CHECKED && (g < 0 || g >= d.G || b < 0 || b >= it.ncols)) { flag_bounds(d.dstatus); return cmk(0.0, 0.0); }
  if (!CIN) {
    const int own = (int)tab[d.geo_off + 4 * g];
    if (own != col_side(d, it.col0 + b)) return cmk(0.0, 0.0);
    return cmk(ws[it.xi_off + (long long)g * it.ncols + b], 0.0);
  }
  const double2 v = xi_user[it.io_off + (long long)b * d.G + g];
  return cmk(v.x, v.y);
}


// Deterministic sum of one double per thread of a (32 x BY) block; thread (0, 0) gets it.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double *sh) {
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
  sh[t] = v;
  __syncthreads();
#pragma unroll
  for (int s = NT / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  return sh[0];
}

// Bit reversal of the lg low bits of j.
__device__ __forceinline__ int brev_lg(int j, int lg) { return (int)(__brev((unsigned)j) >> (32 - lg)); }

// Radix-2 decimation-in-time FFT with the forward sign, V[k] = sum_n x[n] e^{-2 pi i n k / L},
// of nf sequences of length L = 2^lg (4 <= L <= 2 Nx) stored one after another in shared memory
// with their inputs in bit-reversed order; the output is in natural order. Twiddles come from
// the sine table sn[j] = sin(pi j / Nx), j < 2 Nx (cos(pi j / Nx) = sn[j + Nx/2]). The first
// two stages (twiddles 1 and -i) take no multiplies. Called by every thread of the block.
__device__ __forceinline__ void fft_r2_stages(double2 *sm, int nf, int Nx, int lg, const double *sn) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int hl = lg - 1, nb = nf << hl;  // butterflies per stage
  for (int t = tid; t < nb; t += nt) {   // stage 0: pairs (2k, 2k+1)
    double2 *S = sm + ((t >> hl) << lg) + 2 * (t & ((1 << hl) - 1));
    const double2 a = S[0], c = S[1];
    S[0] = make_double2(a.x + c.x, a.y + c.y);
    S[1] = make_double2(a.x - c.x, a.y - c.y);
  }
  __syncthreads();
  for (int t = tid; t < nb; t += nt) {   // stage 1: twiddles 1, -i
    const int k = t & ((1 << hl) - 1), j = k & 1;
    double2 *S = sm + ((t >> hl) << lg) + ((k >> 1) << 2) + j;
    const double2 a = S[0], c = S[2];
    const double2 bb = j ? make_double2(c.y, -c.x) : c;
    S[0] = make_double2(a.x + bb.x, a.y + bb.y);
    S[2] = make_double2(a.x - bb.x, a.y - bb.y);
  }
  __syncthreads();
  for (int st = 2; st < lg; ++st) {
    const int half = 1 << st, span = Nx >> st;  // twiddle e^{-i pi j / half} = e^{-i pi (j span) / Nx}
    for (int t = tid; t < nb; t += nt) {
      const int k = t & ((1 << hl) - 1), j = k & (half - 1);
      double2 *S = sm + ((t >> hl) << lg) + ((k >> st) << (st + 1)) + j;
      const int jj = j * span;
      const double wr = sn[jj + (Nx >> 1)], wi = -sn[jj];
      const double2 a = S[0], c = S[half];
      const double br = fma(wr, c.x, -wi * c.y), bi = fma(wr, c.y, wi * c.x);
      S[0] = make_double2(a.x + br, a.y + bi);
      S[half] = make_double2(a.x - br, a.y - bi);
    }
    __syncthreads();
  }
}


// ---------------------------------------------------------------- DST-I by a length-N FFT
// F_q = sum_{j=1}^{N-1} x_j sin(pi q j / N), q = 1 .. N-1, for complex x and N = 2^lg, from one
// complex FFT of length N (the odd extension would take one of length 2N). With s_j = sin(pi j/N)
// the twisted sequence y_0 = 0, y_j = s_j (x_j + x_{N-j}) + (x_j - x_{N-j}) / 2 has the DFT
// C_k = sum_j y_j e^{-2 pi i j k / N} with
//   F_{2k} = (i/2) (C_k - C_{N-k}),   F_1 = C_0 / 2,   F_{2k+1} = F_{2k-1} + (C_k + C_{N-k}) / 2:
// the part of y symmetric under j -> N - j gives cosine sums, and 2 sin(pi j/N) cos(2 pi j k/N)
// = sin(pi j (2k+1)/N) - sin(pi j (2k-1)/N) makes them differences of consecutive odd outputs;
// the antisymmetric part gives the sine sums at the even outputs. The odd outputs are a prefix
// sum over k (a tree scan: rounding grows like log N). This is the classical reduction of the
// sine transform to a real-input FFT of the same length (Press, Teukolsky, Vetterling and
// Flannery, Numerical Recipes, the section on the fast sine transform), applied here to
// complex data with a full complex FFT, the running sum done as a segmented warp scan.

// y_j and y_{N-j} from the pair xa = x_j, xb = x_{N-j} (j = 1 .. N/2 - 1)
__device__ __forceinline__ void dst1_twist(cplx xa, cplx xb, double s, cplx &ya, cplx &yb) {
  const cplx p = cadd(xa, xb), m = csub(xa, xb);
  ya = cmk(fma(s, p.re, 0.5 * m.re), fma(s, p.im, 0.5 * m.im));
  yb = cmk(fma(s, p.re, -0.5 * m.re), fma(s, p.im, -0.5 * m.im));
}

// From C (nseq transforms of length N, stride N) to F[f N + q] = F_q (q = 1 .. N-1; F[f N] is
// not written). nseq N / 2 must be a multiple of the block size (256 threads): the FFT kernels
// use nseq = P / (2N), or 1 when 2N >= P, with P = 1024, 2048 or 4096 points per block (the plan
// accepts no other), so nseq N / 2 is P / 4 or N / 2 >= 256, a power of two. tot: shared scratch
// of nseq N / 64 <= 32 values. Called by every thread of the block.
__device__ __forceinline__ void dst1_post(const double2 *C, double2 *F, int nseq, int N, double2 *tot) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  const int H = N >> 1, E = nseq * H, lane = tid & 31;
  const int W = H < 32 ? H : 32;   // scan segment in a warp: a whole sequence, or 32 of its terms
  for (int e0 = 0; e0 < E; e0 += nt) {
    const int e = e0 + tid, f = e / H, k = e - f * H;
    const double2 *Cf = C + (long long)f * N;
    double2 *Ff = F + (long long)f * N;
    const double2 a = Cf[k], c = Cf[k == 0 ? 0 : N - k];
    if (k > 0) Ff[2 * k] = make_double2(-0.5 * (a.y - c.y), 0.5 * (a.x - c.x));
    double2 t = k == 0 ? make_double2(0.5 * a.x, 0.5 * a.y) : make_double2(0.5 * (a.x + c.x), 0.5 * (a.y + c.y));
    for (int off = 1; off < W; off <<= 1) {   // inclusive scan within the segment
      const double ux = __shfl_up_sync(0xffffffffu, t.x, off, W), uy = __shfl_up_sync(0xffffffffu, t.y, off, W);
      if ((lane & (W - 1)) >= off) { t.x += ux; t.y += uy; }
    }
    Ff[2 * k + 1] = t;
    if (H > 32 && lane == 31) tot[e >> 5] = t;   // total of this 32-term chunk
  }
  if (H <= 32) { __syncthreads(); return; }
  __syncthreads();
  for (int e0 = 0; e0 < E; e0 += nt) {   // add the totals of the sequence's earlier chunks
    const int e = e0 + tid, f = e / H, k = e - f * H;
    const int c = e >> 5, cfirst = (f * H) >> 5;
    if (c == cfirst) continue;
    double sx = 0.0, sy = 0.0;
    for (int cc = cfirst; cc < c; ++cc) { sx += tot[cc].x; sy += tot[cc].y; }
    double2 *o = F + (long long)f * N + 2 * k + 1;
    *o = make_double2(o->x + sx, o->y + sy);
  }
  __syncthreads();
}

}  // namespace mdp
