// Dense complex linear algebra of the coupled subdomain system (Section 3.5, steps 2(b)-(c): the
// least-squares solve by QR and the triangular solve c = R^{-1} Q^H F), on the GPU in FP64
// (CUDA, sm_103a).
//
// Householder QR. A is column-major m x (n + nrhs). For k = 0 .. n-1 the reflector
// H_k = I - tau_k v_k v_k^H (v_k(k) = 1, v_k zero above k) maps column k below the diagonal onto
// beta_k e_k with beta_k real, and H_k^H is applied to every column right of k, including the
// nrhs right-hand sides: on return the upper triangle of the first n columns is R, the
// reflectors sit below it, tau holds tau_k, and the last nrhs columns hold Q^H b. The reflector
// is the textbook one: with x = A(k:m, k), alpha = x(0),
//   beta = -sign(Re alpha) ||x||,  tau = (beta - alpha) / beta,  v = x / (alpha - beta), v(0) = 1.
//
// GB300 has 2 FP64 FMA lanes per clock per SM, shared by its 4 sub-partitions: one warp reaches
// a quarter of that, and every FP64 add of a reduction costs as much as a useful FMA. A panel of
// reflectors factored inside one SM (the blocked LAPACK form) would run its O(m n nb) panel
// flops at 1/152 of the machine. Here each column operation is done by one CTA of 4 warps (one
// per sub-partition), and the columns are spread over all SMs:
//   - one cooperative launch of persistent CTAs, at most one per SM (every CTA resident);
//     column g of the batch belongs to CTA g mod G and stays in its shared memory (in global
//     memory when the CTA's columns do not fit);
//   - each CTA keeps, per owned column, the number of reflectors applied to it, and repeatedly
//     takes the owned column with the smallest index whose next reflector is published (so the
//     column that forms the next reflector goes first, and the other columns catch up while it
//     waits), together with up to 3 more of its columns waiting for the same reflector;
//   - a column that needs only H_k before forming reflector k+1 takes the fused step: one pass
//     sums conj(v_k) a and |a|^2, one reduction (a warp reduce-scatter, then the 4 warps'
//     totals), the updated column's norm below row k+1 from
//     ||a - s v||^2 = ||a||^2 - 2 Re(conj(s) v^H a) + |s|^2 ||v||^2 with
//     ||v||^2 = 2 Re(tau) / |tau|^2 for a Householder vector (if cancellation could cost more
//     than two bits the updated column is summed again instead), then one pass that updates
//     the column, scales it into v_{k+1}, and writes it to global memory, published by a
//     release store of k + 2 to the matrix's progress counter;
//   - other columns take a dot pass, one reduction and an update pass per reflector, v_k read
//     from L2 into registers once per pass (rows beyond the register cache are read again).
// Every wait is on a published counter and bounded. The chain of a matrix depends only on its
// own earlier reflectors, so with every CTA resident the waits end. Reductions run in a fixed
// order: the result does not depend on timing.
#include "kernels_common.cuh"

#include "mdp.h"

namespace mdp {
namespace {

constexpr int kQrThreads = 128;                    // 4 warps: one per SM sub-partition
constexpr int kQrChunk = 4;                        // columns per fused dot / update pass
constexpr int kQrRv = 28;                          // rows per thread of the register cache of v
constexpr long long kQrWaitCycles = 4000000000LL;  // about 2 s at the maximum SM clock

struct QrArgs {
  int batch, m, n, ncols;     // ncols = n + nrhs columns per matrix
  double2 *A;
  long long lda, stride;
  double2 *tau;               // [batch][n]
  int *progress;              // [batch]: reflectors published so far (zeroed before the launch)
  int *status;                // [2]: sticky status word, abort flag
  int G;                      // CTAs
  int Gb;                     // CTAs per matrix (each CTA owns columns of one matrix), or 0: each CTA owns whole matrices
  int slots;                  // most columns owned by one CTA
};

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// a - v s (complex), with explicit FMAs so that every thread that evaluates it gets the same bits
__device__ __forceinline__ double2 sub_vs(double2 a, double2 v, double2 s) {
  return make_double2(a.x - fma(v.x, s.x, -v.y * s.y), a.y - fma(v.x, s.y, v.y * s.x));
}

// Reduce-scatter of 8 values over a warp: lane l returns the warp's total of value (l >> 2) & 7
// (9 adds per lane instead of the 40 of eight butterflies).
__device__ __forceinline__ double warp_rs8(const double (&v)[8]) {
  const int lane = threadIdx.x & 31;
  double a[4], b[2];
  const bool h16 = lane & 16, h8 = lane & 8, h4 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double keep = h16 ? v[q + 4] : v[q], send = h16 ? v[q] : v[q + 4];
    a[q] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const double keep = h8 ? a[q + 2] : a[q], send = h8 ? a[q] : a[q + 2];
    b[q] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const double keep = h4 ? b[1] : b[0], send = h4 ? b[0] : b[1];
  double c = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  c += __shfl_xor_sync(0xffffffffu, c, 2);
  c += __shfl_xor_sync(0xffffffffu, c, 1);
  return c;
}

// Block totals of the threads' v[0..8): fin[0..8) in shared memory, visible to every thread on
// return (two barriers; consecutive calls may reuse red and fin).
__device__ __forceinline__ void block_sum8(const double (&v)[8], double *red, double *fin) {
  const double t = warp_rs8(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if ((lane & 3) == 0) red[warp * 8 + (lane >> 2)] = t;
  __syncthreads();
  if (threadIdx.x < 8) {
    const int j = threadIdx.x;
    fin[j] = (red[j] + red[8 + j]) + (red[16 + j] + red[24 + j]);
  }
  __syncthreads();
}

// The reflector of a column from alpha = x(c) and xn2 = ||x(c+1:)||^2: beta, tau, and
// inv = 1 / (alpha - beta); false if the column is already beta e_c with beta real (H = I).
// With g = beta - Re(alpha) (no cancellation: beta has the sign opposite to Re(alpha)),
// tau = (g - i Im(alpha)) / beta and inv = (-g - i Im(alpha))^* / (g^2 + Im(alpha)^2): two
// independent divisions.
__device__ __forceinline__ bool reflector_of(double2 a, double xn2, double &beta, double2 &tau, double2 &inv) {
  if (xn2 == 0.0 && a.y == 0.0) {
    beta = a.x;
    tau = make_double2(0.0, 0.0);
    inv = make_double2(0.0, 0.0);
    return false;
  }
  const double nrm = sqrt(fma(a.x, a.x, fma(a.y, a.y, xn2)));
  beta = a.x >= 0.0 ? -nrm : nrm;
  const double g = beta - a.x;
  const double rb = 1.0 / beta, rd = 1.0 / fma(g, g, a.y * a.y);
  inv = make_double2(-g * rd, -a.y * rd);   // conj(alpha - beta) / |alpha - beta|^2
  tau = make_double2(g * rb, -a.y * rb);
  return true;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// One reflector applied to up to 4 owned columns of one matrix (plain update), or the fused
// step on the column that forms the next reflector (crit): see the file comment.
struct QrItem {
  int kind;        // 0: work, 1: all done, 2: abort
  int b, j, crit, nc;
  int slot[4];
};

template <bool SMEM>
__global__ void __launch_bounds__(kQrThreads) k_qr_cta(QrArgs q) {
  extern __shared__ __align__(16) double2 qsm[];   // [slots][m] owned columns, then [slots] ints
  __shared__ double red[32], fin[8];
  __shared__ double2 vk1s;
  __shared__ QrItem items[2];   // alternating: the next item is chosen while the last is still read
  int par = 0;
  const int m = q.m, C = q.ncols, G = q.G, me = blockIdx.x, tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  // owned columns: with Gb > 0, matrix me / Gb, columns c = me % Gb + s Gb; else matrices
  // b = me + (s / C) G, all their columns
  const int nslots = q.Gb > 0 ? (C - me % q.Gb + q.Gb - 1) / q.Gb
                              : (me < q.batch ? (q.batch - me + G - 1) / G : 0) * C;
  auto slot_bc = [&](int s, int &b, int &c) {
    if (q.Gb > 0) {
      b = me / q.Gb;
      c = me % q.Gb + s * q.Gb;
    } else {
      b = me + (s / C) * G;
      c = s % C;
    }
  };
  int *nxt = reinterpret_cast<int *>(qsm + (SMEM ? (long long)q.slots * m : 0));   // reflectors applied, per slot

  auto gcol = [&](int b, int c) -> double2 * { return q.A + (long long)b * q.stride + (long long)c * q.lda; };
  auto col_of_slot = [&](int s) -> double2 * {
    int b, c;
    slot_bc(s, b, c);
    if (SMEM) return qsm + (long long)s * m;
    return gcol(b, c);
  };
  auto publish = [&](int b, int c) {   // after every thread wrote its part of column (b, c)
    __threadfence();
    __syncthreads();
    if (tid == 0) st_release_gpu(q.progress + b, c + 1);
  };

  for (int s = tid; s < nslots; s += kQrThreads) nxt[s] = 0;
  if (SMEM) {
    for (int s = 0; s < nslots; ++s) {
      int b, c;
      slot_bc(s, b, c);
      const double2 *src = gcol(b, c);
      for (int i = tid; i < m; i += kQrThreads) qsm[(long long)s * m + i] = src[i];
    }
  }
  __syncthreads();
  // the first reflector of every matrix whose column 0 this CTA owns
  for (int s = 0; s < nslots; ++s) {
    int b, c;
    slot_bc(s, b, c);
    if (c != 0) continue;
    double2 *x = col_of_slot(s);
    const double2 a0 = x[0];
    double p[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int i = 1 + tid; i < m; i += kQrThreads) p[0] = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, p[0]));
    block_sum8(p, red, fin);
    double beta;
    double2 t, inv;
    const bool refl = reflector_of(a0, fin[0], beta, t, inv);
    double2 *gc = gcol(b, 0);
    for (int i = tid; i < m; i += kQrThreads) {
      double2 a = x[i];
      if (i == 0) a = make_double2(beta, 0.0);
      else if (refl) a = cmul(a, inv);
      if (SMEM) x[i] = a;
      gc[i] = a;
    }
    if (tid == 0) q.tau[(long long)b * q.n] = t;
    publish(b, 0);
  }

  while (true) {
    // warp 0 picks the next item: among the owned columns whose next reflector is published, the
    // one closest to forming its matrix's next reflector (c - published, then matrix, then
    // column); more columns of that matrix waiting for the same reflector share the pass unless
    // the first one forms the next reflector
    QrItem &item = items[par];
    par ^= 1;
    if (warp == 0) {
      __syncwarp();   // tid 0's updates of nxt
      const long long t0 = clock64();
      while (true) {
        long long best = 0x7fffffffffffffffLL;
        int pending = 0;
        for (int s = lane; s < nslots; s += 32) {
          int b, c;
          slot_bc(s, b, c);
          const int j = nxt[s], tg = c < q.n ? c : q.n;
          if (j < tg) {
            pending = 1;
            const int pub = ld_acquire_gpu(q.progress + b);
            if (pub > j) {
              const long long key = ((long long)(c - pub) << 42) | ((long long)b << 21) | s;
              best = key < best ? key : best;
            }
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          const long long other = __shfl_xor_sync(0xffffffffu, best, o);
          best = other < best ? other : best;
        }
        const bool any_pending = __any_sync(0xffffffffu, pending);
        if (best != 0x7fffffffffffffffLL || !any_pending) {
          if (lane == 0) {
            if (best == 0x7fffffffffffffffLL) {
              item.kind = 1;
            } else {
              const int s0 = (int)(best & ((1 << 21) - 1));
              int b, c;
              slot_bc(s0, b, c);
              const int j = nxt[s0];
              item.kind = 0;
              item.b = b;
              item.j = j;
              item.crit = c < q.n && j == c - 1;
              item.slot[0] = s0;
              int nc = 1;
              if (!item.crit)
                for (int s2 = 0; s2 < nslots && nc < kQrChunk; ++s2) {
                  int b2, c2;
                  slot_bc(s2, b2, c2);
                  const int tg2 = c2 < q.n ? c2 : q.n;
                  if (s2 != s0 && b2 == b && nxt[s2] == j && j < tg2 && !(c2 < q.n && j == c2 - 1)) item.slot[nc++] = s2;
                }
              item.nc = nc;
            }
          }
          break;
        }
        const int ab = ld_acquire_gpu(q.status + 1);
        const bool late = __shfl_sync(0xffffffffu, clock64() - t0 > kQrWaitCycles, 0);
        if (__any_sync(0xffffffffu, ab != 0) || late) {
          if (lane == 0) {
            if (late) {
              atomicCAS(q.status, 0, (int)MDP_ERR_TIMEOUT);
              atomicExch(q.status + 1, 1);
            }
            item.kind = 2;
          }
          break;
        }
        __nanosleep(64);
      }
    }
    __syncthreads();
    const QrItem it = item;
    if (it.kind == 2) return;
    if (it.kind == 1) break;
    const int b = it.b, k = it.j;
    (void)ld_acquire_gpu(q.progress + b);   // each thread's own acquire of the published reflector
    const double2 *vg = gcol(b, k);
    const double2 t = __ldcg(q.tau + (long long)b * q.n + k);
    const bool apply = t.x != 0.0 || t.y != 0.0;
    const int nu = min(kQrRv, (m - k + kQrThreads - 1) / kQrThreads);
    double2 vr[kQrRv];   // v(k + tid + 128 u)
#pragma unroll
    for (int u = 0; u < kQrRv; ++u) {
      const int i = k + tid + kQrThreads * u;
      vr[u] = u >= nu || i >= m ? make_double2(0.0, 0.0) : (i == k ? make_double2(1.0, 0.0) : __ldcg(vg + i));
    }
    if (it.crit) {
      // apply H_k to column k+1 and form reflector k+1 from it
      double2 *x = col_of_slot(it.slot[0]);
      const double2 a0 = x[k], a1 = x[k + 1];   // read before any thread changes the column
      const double2 v1 = apply ? vr[0] : make_double2(0.0, 0.0);
      // ||v||^2 = 2 Re(tau) / |tau|^2 for a Householder vector: its division overlaps the pass
      const double vn = apply ? 2.0 * t.x / fma(t.x, t.x, t.y * t.y) : 0.0;
      double p[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // v^H a and ||a||^2 over rows > k+1
#pragma unroll
      for (int u = 0; u < kQrRv; ++u) {
        if (u >= nu) break;
        const int i = k + tid + kQrThreads * u;
        if (i > k + 1 && i < m) {
          const double2 a = x[i], v = vr[u];
          p[0] = fma(v.x, a.x, fma(v.y, a.y, p[0]));
          p[1] = fma(v.x, a.y, fma(-v.y, a.x, p[1]));
          p[2] = fma(a.x, a.x, fma(a.y, a.y, p[2]));
        }
      }
      for (int i = k + tid + kQrThreads * kQrRv; i < m; i += kQrThreads) {
        const double2 a = x[i], v = __ldcg(vg + i);
        p[0] = fma(v.x, a.x, fma(v.y, a.y, p[0]));
        p[1] = fma(v.x, a.y, fma(-v.y, a.x, p[1]));
        p[2] = fma(a.x, a.x, fma(a.y, a.y, p[2]));
      }
      if (tid == 1) vk1s = v1;   // v(k+1) is vr[0] of the thread that holds row k+1
      block_sum8(p, red, fin);   // its barriers also publish vk1s
      const double2 vk1 = vk1s;
      const double2 d = make_double2(fin[0], fin[1]);
      const double s2 = fin[2];
      // w = v^H a over rows >= k: v(k) = 1, plus row k+1
      const double2 w = make_double2(d.x + a0.x + fma(vk1.x, a1.x, vk1.y * a1.y),
                                     d.y + a0.y + fma(vk1.x, a1.y, -vk1.y * a1.x));
      const double2 s = apply ? make_double2(fma(t.x, w.x, t.y * w.y), fma(t.x, w.y, -t.y * w.x))   // conj(tau) w
                              : make_double2(0.0, 0.0);
      const double2 alpha = sub_vs(a1, vk1, s);
      double xn2 = s2;
      bool exact = true;
      if (apply) {
        const double vn2 = vn - 1.0 - fma(vk1.x, vk1.x, vk1.y * vk1.y);   // ||v(k+2:)||^2
        const double sd = fma(s.x, d.x, s.y * d.y);                      // Re(conj(s) d)
        xn2 = fma(fma(s.x, s.x, s.y * s.y), vn2, fma(-2.0, sd, s2));
        exact = s2 > 0.0 && xn2 >= 0.25 * s2;
      }
      if (!exact) {   // cancellation: update, summing the updated column's norm in the same pass
        double pp[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int u = 0; u < kQrRv; ++u) {
          if (u >= nu) break;
          const int i = k + tid + kQrThreads * u;
          if (i < m) {
            const double2 a = sub_vs(x[i], vr[u], s);
            x[i] = a;
            if (i > k + 1) pp[0] = fma(a.x, a.x, fma(a.y, a.y, pp[0]));
          }
        }
        for (int i = k + tid + kQrThreads * kQrRv; i < m; i += kQrThreads) {
          const double2 a = sub_vs(x[i], __ldcg(vg + i), s);
          x[i] = a;
          pp[0] = fma(a.x, a.x, fma(a.y, a.y, pp[0]));
        }
        block_sum8(pp, red, fin);
        xn2 = fin[0];
      }
      double beta;
      double2 tn, inv;
      const bool refl = reflector_of(alpha, xn2, beta, tn, inv);
      const double2 si = cmul(s, inv);   // (a - s v) inv = a inv - (s inv) v
      double2 *gc = gcol(b, k + 1);
      if (SMEM)   // rows of R above row k are final: copy them out
        for (int i = tid; i < k; i += kQrThreads) gc[i] = x[i];
#pragma unroll
      for (int u = 0; u < kQrRv; ++u) {
        if (u >= nu) break;
        const int i = k + tid + kQrThreads * u;
        if (i < m) {
          double2 a;
          if (i == k + 1) a = make_double2(beta, 0.0);
          else if (i == k || !refl) a = exact ? sub_vs(x[i], vr[u], s) : x[i];
          else a = exact ? sub_vs(cmul(x[i], inv), vr[u], si) : cmul(x[i], inv);
          if (SMEM) x[i] = a;
          gc[i] = a;
        }
      }
      for (int i = k + tid + kQrThreads * kQrRv; i < m; i += kQrThreads) {
        double2 a;
        if (!refl) a = exact ? sub_vs(x[i], __ldcg(vg + i), s) : x[i];
        else a = exact ? sub_vs(cmul(x[i], inv), __ldcg(vg + i), si) : cmul(x[i], inv);
        if (SMEM) x[i] = a;
        gc[i] = a;
      }
      if (tid == 0) {
        q.tau[(long long)b * q.n + k + 1] = tn;
        nxt[it.slot[0]] = k + 1;
      }
      publish(b, k + 1);
      continue;
    }
    const int nc = it.nc;
    double2 *cols[kQrChunk];
#pragma unroll
    for (int jj = 0; jj < kQrChunk; ++jj) cols[jj] = jj < nc ? col_of_slot(it.slot[jj]) : nullptr;
    if (apply) {
      double p[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};   // v^H a of each column of the pass
#pragma unroll
      for (int u = 0; u < kQrRv; ++u) {
        if (u >= nu) break;
        const int i = k + tid + kQrThreads * u;
        if (i < m) {
          const double2 v = vr[u];
#pragma unroll
          for (int jj = 0; jj < kQrChunk; ++jj)
            if (jj < nc) {
              const double2 a = cols[jj][i];
              p[2 * jj] = fma(v.x, a.x, fma(v.y, a.y, p[2 * jj]));
              p[2 * jj + 1] = fma(v.x, a.y, fma(-v.y, a.x, p[2 * jj + 1]));
            }
        }
      }
      for (int i = k + tid + kQrThreads * kQrRv; i < m; i += kQrThreads) {
        const double2 v = __ldcg(vg + i);
#pragma unroll
        for (int jj = 0; jj < kQrChunk; ++jj)
          if (jj < nc) {
            const double2 a = cols[jj][i];
            p[2 * jj] = fma(v.x, a.x, fma(v.y, a.y, p[2 * jj]));
            p[2 * jj + 1] = fma(v.x, a.y, fma(-v.y, a.x, p[2 * jj + 1]));
          }
      }
      block_sum8(p, red, fin);
      double2 sj[kQrChunk];
#pragma unroll
      for (int jj = 0; jj < kQrChunk; ++jj)
        sj[jj] = make_double2(fma(t.x, fin[2 * jj], t.y * fin[2 * jj + 1]), fma(t.x, fin[2 * jj + 1], -t.y * fin[2 * jj]));
#pragma unroll
      for (int u = 0; u < kQrRv; ++u) {
        if (u >= nu) break;
        const int i = k + tid + kQrThreads * u;
        if (i < m) {
#pragma unroll
          for (int jj = 0; jj < kQrChunk; ++jj)
            if (jj < nc) cols[jj][i] = sub_vs(cols[jj][i], vr[u], sj[jj]);
        }
      }
      for (int i = k + tid + kQrThreads * kQrRv; i < m; i += kQrThreads) {
        const double2 v = __ldcg(vg + i);
#pragma unroll
        for (int jj = 0; jj < kQrChunk; ++jj)
          if (jj < nc) cols[jj][i] = sub_vs(cols[jj][i], v, sj[jj]);
      }
    }
    if (tid == 0)
      for (int jj = 0; jj < nc; ++jj) nxt[it.slot[jj]] = k + 1;
  }
  if (SMEM) {   // the right-hand sides (the reflector columns were written when published)
    for (int s = 0; s < nslots; ++s) {
      int b, c;
      slot_bc(s, b, c);
      if (c < q.n) continue;
      double2 *dst = gcol(b, c);
      for (int i = tid; i < m; i += kQrThreads) dst[i] = qsm[(long long)s * m + i];
    }
  }
}

// ---- triangular solve --------------------------------------------------------------------------
// R x = b (back substitution) or R^H x = b (forward substitution), R upper triangular,
// column-major with leading dimension ldr (only i <= j is read). One CTA per right-hand side,
// the vector in shared memory; blocks of 32 rows: the block's 32 x 32 triangle is staged in
// shared memory by all threads (coalesced), warp 0 forms the 32 reciprocals of its diagonal at
// once and solves the block with shuffles, then all threads subtract the block's contribution
// from the rows still to solve, one row per thread (loads issued 8 at a time, no reductions).
constexpr int kTrThreads = 256;

__device__ __forceinline__ double2 crcp(double2 d) {   // 1 / d
  const double den = fma(d.x, d.x, d.y * d.y);
  return make_double2(d.x / den, -d.y / den);
}

template <bool CT>
__global__ void __launch_bounds__(kTrThreads) k_trsv(int n, const double2 *__restrict__ R, long long ldr,
                                                     double2 *B, long long ldb) {
  extern __shared__ __align__(16) double2 xs[];
  __shared__ double2 T[32][33];   // the diagonal block: T[col][row] = R(i0 + row, i0 + col)
  double2 *bcol = B + (long long)blockIdx.x * ldb;
  for (int i = threadIdx.x; i < n; i += kTrThreads) xs[i] = bcol[i];
  const int nblk = (n + 31) / 32, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = 0; t < nblk; ++t) {
    const int bi = CT ? t : nblk - 1 - t;
    const int i0 = bi * 32, w = min(32, n - i0);
    for (int e = threadIdx.x; e < 32 * 32; e += kTrThreads) {
      const int cc = e >> 5, rr = e & 31;   // rr fastest: a column of the block, coalesced
      T[cc][rr] = cc < w && rr <= cc ? R[(long long)(i0 + cc) * ldr + i0 + rr] : make_double2(0.0, 0.0);
    }
    __syncthreads();   // T, and the previous block's updates of xs
    if (warp == 0) {
      const int r = i0 + lane;
      double2 v = lane < w ? xs[r] : make_double2(0.0, 0.0);
      const double2 dinv = lane < w ? crcp(T[lane][lane]) : make_double2(0.0, 0.0);
      if (!CT) {
        for (int j = w - 1; j >= 0; --j) {
          if (lane == j) v = cmul(v, dinv);
          const double2 xj = make_double2(__shfl_sync(0xffffffffu, v.x, j), __shfl_sync(0xffffffffu, v.y, j));
          if (lane < j) {
            const double2 a = T[j][lane];   // R(r, i0 + j)
            v.x -= fma(a.x, xj.x, -a.y * xj.y);
            v.y -= fma(a.x, xj.y, a.y * xj.x);
          }
        }
      } else {
        const double2 dinvc = make_double2(dinv.x, -dinv.y);   // 1 / conj(d)
        for (int j = 0; j < w; ++j) {
          if (lane == j) v = cmul(v, dinvc);
          const double2 xj = make_double2(__shfl_sync(0xffffffffu, v.x, j), __shfl_sync(0xffffffffu, v.y, j));
          if (lane > j && lane < w) {
            const double2 a = T[lane][j];   // R(i0 + j, r); L(r, i0 + j) = conj of it
            v.x -= fma(a.x, xj.x, a.y * xj.y);
            v.y -= fma(a.x, xj.y, -a.y * xj.x);
          }
        }
      }
      if (lane < w) xs[r] = v;
    }
    __syncthreads();
    if (!CT) {   // rows above the block: thread per row, R(r, i0 + j) coalesced over r
      for (int r = threadIdx.x; r < i0; r += kTrThreads) {
        double sx = 0.0, sy = 0.0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
          if (j < w) {
            const double2 a = R[(long long)(i0 + j) * ldr + r];
            const double2 x = xs[i0 + j];
            sx = fma(a.x, x.x, fma(-a.y, x.y, sx));
            sy = fma(a.x, x.y, fma(a.y, x.x, sy));
          }
        }
        xs[r].x -= sx;
        xs[r].y -= sy;
      }
    } else {     // rows below the block: thread per row, conj(R(i0 + j, r)) from column r of R
      for (int r = i0 + w + threadIdx.x; r < n; r += kTrThreads) {
        const double2 *rc = R + (long long)r * ldr + i0;
        double sx = 0.0, sy = 0.0;
#pragma unroll 8
        for (int j = 0; j < 32; ++j) {
          if (j < w) {
            const double2 a = rc[j];
            const double2 x = xs[i0 + j];
            sx = fma(a.x, x.x, fma(a.y, x.y, sx));
            sy = fma(a.x, x.y, fma(-a.y, x.x, sy));
          }
        }
        xs[r].x -= sx;
        xs[r].y -= sy;
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += kTrThreads) bcol[i] = xs[i];
}

// ---- small complex matrix product --------------------------------------------------------------
// C = op(A) op(B) (+ C), op = identity or complex conjugate, every operand given by a row and a
// column stride (so transposes are views). 16 x 16 outputs per block, the 16 x 16 operand tiles
// staged in shared memory; each output sums its k products in order.
__global__ void __launch_bounds__(256) k_cmatmul(int m, int n, int k, const double2 *__restrict__ A, long long rsa,
                                                 long long csa, int conja, const double2 *__restrict__ B,
                                                 long long rsb, long long csb, int conjb, double2 *C,
                                                 long long rsc, long long csc, int accumulate) {
  __shared__ double2 As[16][17], Bs[16][17];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  const double sa = conja ? -1.0 : 1.0, sb = conjb ? -1.0 : 1.0;
  double cx = 0.0, cy = 0.0;
  for (int l0 = 0; l0 < k; l0 += 16) {
    const int ac = l0 + tx, br = l0 + ty;
    double2 a = make_double2(0.0, 0.0), bb = make_double2(0.0, 0.0);
    if (row < m && ac < k) a = A[(long long)row * rsa + (long long)ac * csa];
    if (br < k && col < n) bb = B[(long long)br * rsb + (long long)col * csb];
    As[ty][tx] = make_double2(a.x, sa * a.y);
    Bs[ty][tx] = make_double2(bb.x, sb * bb.y);
    __syncthreads();
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      const double2 x = As[ty][l], y = Bs[l][tx];
      cx = fma(x.x, y.x, fma(-x.y, y.y, cx));
      cy = fma(x.x, y.y, fma(x.y, y.x, cy));
    }
    __syncthreads();
  }
  if (row < m && col < n) {
    double2 *c = C + (long long)row * rsc + (long long)col * csc;
    if (accumulate) {
      const double2 o = *c;
      cx += o.x;
      cy += o.y;
    }
    *c = make_double2(cx, cy);
  }
}

// Cooperative launch shape of k_qr_cta: at most one CTA per SM, so that consecutive columns of a
// matrix land on different SMs. A batch of at most n_sm matrices gives each matrix its own Gb
// CTAs (a CTA's columns then share passes); a larger batch gives each CTA whole matrices. The
// columns stay in shared memory when they fit.
struct QrShape {
  int G, Gb, slots;
  bool in_smem;
  size_t smem;
};

bool qr_shape(int batch, int C, int m, int n_sm, QrShape &s) {
  int G, Gb, slots;
  if (batch <= n_sm) {
    Gb = n_sm / batch < C ? n_sm / batch : C;
    G = batch * Gb;
    slots = (C + Gb - 1) / Gb;
  } else {
    G = n_sm;
    Gb = 0;
    slots = (batch + G - 1) / G * C;
  }
  const size_t ints = ((size_t)slots * sizeof(int) + 15) / 16 * 16;
  const size_t smem = (size_t)slots * (size_t)m * sizeof(double2) + ints;
  int per_sm = 0;
  if (smem <= 200 * 1024 &&
      cudaFuncSetAttribute(k_qr_cta<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_cta<true>, kQrThreads, smem) == cudaSuccess &&
      per_sm >= 1) {
    s = QrShape{G, Gb, slots, true, smem};
    return true;
  }
  if (ints > 200 * 1024 ||
      cudaFuncSetAttribute(k_qr_cta<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ints) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_qr_cta<false>, kQrThreads, ints) != cudaSuccess ||
      per_sm < 1)
    return false;
  s = QrShape{G, Gb, slots, false, ints};
  return true;
}

}  // namespace
}  // namespace mdp

extern "C" long long mdp_householder_qr_work_ints(int batch) { return batch < 0 ? 0 : (long long)batch + 2; }

extern "C" mdp_status mdp_householder_qr_batched(int batch, int m, int n, int nrhs, mdp_c64 *A, long long lda,
                                                 long long stride, mdp_c64 *tau, int *work, void *cuda_stream) {
  if (batch < 1 || m < 1 || n < 1 || n > m || nrhs < 0 || !A || !tau || !work || lda < m ||
      (batch > 1 && stride < lda * (long long)(n + nrhs)) || (long long)batch * (n + nrhs) > (1LL << 30))
    return MDP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, n_sm = 0, coop = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess ||
      cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return MDP_ERR_CUDA;
  if (n + nrhs >= (1 << 21) || batch >= (1 << 21)) return MDP_ERR_ARG;   // the scheduler's 21-bit key fields
  mdp::QrShape s{0, 0, 0, false, 0};
  if (!mdp::qr_shape(batch, n + nrhs, m, n_sm, s)) return MDP_ERR_CUDA;
  if (s.slots >= (1 << 21)) return MDP_ERR_ARG;
  if (cudaMemsetAsync(work, 0, sizeof(int) * ((size_t)batch + 2), st) != cudaSuccess) return MDP_ERR_CUDA;
  mdp::QrArgs q{batch, m, n, n + nrhs, reinterpret_cast<double2 *>(A), lda, stride,
                reinterpret_cast<double2 *>(tau), work, work + batch, s.G, s.Gb, s.slots};
  void *args[] = {&q};
  const cudaError_t e =
      s.in_smem ? cudaLaunchCooperativeKernel((const void *)mdp::k_qr_cta<true>, dim3(s.G), dim3(mdp::kQrThreads), args,
                                              s.smem, st)
                : cudaLaunchCooperativeKernel((const void *)mdp::k_qr_cta<false>, dim3(s.G), dim3(mdp::kQrThreads),
                                              args, s.smem, st);
  return e == cudaSuccess ? MDP_OK : MDP_ERR_CUDA;
}

extern "C" mdp_status mdp_householder_qr(int m, int n, int nrhs, mdp_c64 *A, long long lda, mdp_c64 *tau, int *work,
                                         void *cuda_stream) {
  return mdp_householder_qr_batched(1, m, n, nrhs, A, lda, 0, tau, work, cuda_stream);
}

extern "C" mdp_status mdp_triangular_solve(int n, int nrhs, const mdp_c64 *R, long long ldr, int conj_trans,
                                           mdp_c64 *B, long long ldb, void *cuda_stream) {
  if (n < 1 || nrhs < 1 || nrhs > (1 << 30) || !R || !B || ldr < n || ldb < n ||
      (size_t)n * sizeof(double2) > 227 * 1024)
    return MDP_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t smem = (size_t)n * sizeof(double2);
  const double2 *r = reinterpret_cast<const double2 *>(R);
  double2 *b = reinterpret_cast<double2 *>(B);
  if (conj_trans) {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(mdp::k_trsv<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return MDP_ERR_CUDA;
    mdp::k_trsv<true><<<nrhs, mdp::kTrThreads, smem, st>>>(n, r, ldr, b, ldb);
  } else {
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(mdp::k_trsv<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return MDP_ERR_CUDA;
    mdp::k_trsv<false><<<nrhs, mdp::kTrThreads, smem, st>>>(n, r, ldr, b, ldb);
  }
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_ERR_CUDA;
}

extern "C" mdp_status mdp_complex_matmul(int m, int n, int k, const mdp_c64 *A, long long rsa, long long csa,
                                         int conja, const mdp_c64 *B, long long rsb, long long csb, int conjb,
                                         mdp_c64 *C, long long rsc, long long csc, int accumulate, void *cuda_stream) {
  if (m < 0 || n < 0 || k < 0 || (m > 0 && n > 0 && !C) || (m > 0 && n > 0 && k > 0 && (!A || !B)) ||
      (m + 15) / 16 > 65535)
    return MDP_ERR_ARG;
  if (m == 0 || n == 0) return MDP_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  mdp::k_cmatmul<<<dim3((n + 15) / 16, (m + 15) / 16), 256, 0, st>>>(
      m, n, k, reinterpret_cast<const double2 *>(A), rsa, csa, conja, reinterpret_cast<const double2 *>(B), rsb, csb,
      conjb, reinterpret_cast<double2 *>(C), rsc, csc, accumulate);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_ERR_CUDA;
}
