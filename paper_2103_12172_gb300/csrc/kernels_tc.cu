// k_inv_cols_tc: the inverse sine transform at the 4 gamma columns of the middle rows
// (Section 3.2.1 / 3.6: the AP solution u(m, n) = (2/Nx) sum_q sin(pi q m/Nx) yhat(q, n), taken
// only where the trace on gamma needs it, Eqs. def_Pgamma and Q_construction) as a contraction
// over the mode index q on the tensor cores, to FP64 accuracy.
//
// For one middle row n and a tile of 64 columns the sums are a product D = A B with
//   A[r][q] = yhat(q, n) of matrix row r = (column, real or imaginary part): 128 rows, K = Nq;
//   B[q][s] = sin(pi q m_s / Nx) for the outputs s (x-centred subdomains: the odd-q and even-q
//            partial sums at m = mlo-1 and mlo, which give all four gamma columns; otherwise the
//            four columns mlo-1, mlo, mhi, mhi+1 directly).
// FP64 accuracy from fp16 operands follows the error-free splitting of Ozaki, Ogita, Oishi and
// Rump (Numer. Algorithms 59, 2012). Every value x of a column becomes a signed fixed-point
// integer V on one scale common to the column: with p set by the column's largest exponent
// (|x| < 2^(p-1)), the FP64 sum y = x + 1.5 2^p stays in the binade of 1.5 2^p, so its bit
// pattern minus that of 1.5 2^p is V = round(x / 2^(p-52)), |V| < 2^51 (one FP64 add per value,
// on a pipe this kernel leaves free). V is written in 7 balanced base-256 digits d_t in
// [-128, 127] (V = sum_t d_t 256^(6-t)): adding 128 to every byte position of V makes each byte
// d_t + 128, so two digits cost a byte permute, a mask and one packed fp16 subtraction, and are
// exact in fp16. B, the sine factors, is cut the same way with the fixed scale of |sin| <= 1,
// once, when the plan is built (a 1 KiB block per 16 modes in the shared-memory operand layout).
// A product of two digits is at most 2^14 in magnitude, so a sum over at most 1024 modes is an
// integer of at most 2^24: exact in the tensor core's FP32 accumulator. That covers Nq <= 2047
// on centred subdomains (each output sums one parity of q) and Nq <= 1023 otherwise. All 7 x 7
// digit products are accumulated: D_t = A_t (B_0 .. B_6), one MMA per A digit (M = 128,
// N = 4 outputs x 8 rows, the 8th of each output zero, K = 16), D in tensor memory (7 x 32 FP32
// columns). The epilogue reads D back, converts every product sum to an integer, adds those of
// equal weight t + u in 64-bit integers and scales them into FP64: the only roundings are the
// truncation of the operands to 54 bits and the final conversions, against FP64's rounding at
// every step of the plain sum.
//
// Work: persistent CTAs (two per SM) walk the tiles (item, middle row, 64 columns) in the same
// order in all their warps. Eight producer warps cut the values into digits and fill 3
// shared-memory stages of 16 modes each (canonical K-major layout without swizzle): each thread
// loads 8 values, coalesced along the column and one stage ahead, and stores one 16-byte
// core-matrix row per digit. A ninth warp issues the MMAs of a stage once its `full` mbarrier
// has all 256 producer arrivals and commits them to the stage's `empty` mbarrier, which the
// producers wait on before refilling it; after the last stage of a tile it commits to `tfull`,
// and waits on `tempty` (every producer has read D) before the next tile overwrites D. Every wait
// has a time limit; a wait that runs out sets the plan's status word to MDP_ERR_TIMEOUT and every
// warp leaves its loop, frees the tensor memory and returns; the two producer halves exchange
// their partial sums through an mbarrier (`xbar`) with the same limit. The scale of a column is the
// largest exponent over its modes and kept rows, which the per-mode sweep (k_tri) records as it
// stores them.
#include "kernels_common.cuh"

namespace mdp {
namespace {

constexpr int TC_PRODUCERS = 256;             // 8 warps: matrix row r = 32 (warp % 4) + lane
constexpr int TC_THREADS = TC_PRODUCERS + 32; // + the MMA warp
constexpr int TC_KC = 16;                     // modes per stage (one MMA K step)
constexpr int TC_STAGES = 3;
constexpr int TC_DIG = 7;                     // balanced base-256 digits of |V| < 2^54
constexpr int TC_A_BYTES = 128 * TC_KC * 2;   // one digit of A: 128 rows x 16 bf16
constexpr int TC_B_BYTES = 32 * TC_KC * 2;    // B: 4 outputs x 8 rows x 16 bf16
constexpr int TC_STAGE_BYTES = TC_DIG * TC_A_BYTES + TC_B_BYTES;
constexpr int TC_TMEM_COLS = 256;             // D: 7 A digits x 32 FP32 columns
constexpr long long TC_WAIT_CYCLES = 4000000000LL;   // about 2 s at the maximum clock

__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  // shared-memory matrix descriptor: start address, leading (K) and stride (M/N) byte offsets of
  // the 8 x 16-byte core matrices, descriptor version 1, no swizzle
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, fp16 A and B, both K-major, N = 32, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_try(unsigned addr, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok) : "r"(addr), "r"(parity) : "memory");
  return ok != 0;
}
// wait for the completion of the phase with parity `parity`, at most TC_WAIT_CYCLES; false when
// the limit ran out or another warp has already given up (*abort)
__device__ __forceinline__ bool mbar_wait(unsigned addr, unsigned parity, volatile int *abort) {
  const long long t0 = clock64();
  while (!mbar_try(addr, parity)) {
    if (*abort) return false;
    if (clock64() - t0 > TC_WAIT_CYCLES) { *abort = 1; return false; }
  }
  return true;
}
__device__ __forceinline__ void mbar_arrive(unsigned addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_commit(unsigned mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

// 32 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(unsigned taddr, float *v) {
  unsigned r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// The bit pattern of the magic constant 1.5 2^p for a column whose largest biased exponent is E:
// p = E - 1021 makes every value of the column smaller than 2^(p-1) in magnitude.
__device__ __forceinline__ long long magic_bits(int E) {
  return ((long long)(min(max(E, 0), 2044) + 2) << 52) | (1LL << 51);
}
// x on the column's fixed-point scale plus 0x0080808080808080 (bytes: balanced digits + 128):
// the bits of x + 1.5 2^p minus (the bits of 1.5 2^p - 0x0080808080808080) = cb. As (hi, lo).
__device__ __forceinline__ void digits52(double x, double magic, long long cb, unsigned &hi, unsigned &lo) {
  const long long w = __double_as_longlong(x + magic) - cb;
  hi = (unsigned)((unsigned long long)w >> 32);
  lo = (unsigned)w;
}
// The same fixed-point value by integer operations only (for the values the FP64 pipe does not
// take): the significand m (53 bits) of x, exponent e, gives V = trunc(m 2^(e - E - 2)) on the
// column scale of magic_bits(E); zeros and subnormals give 0 (their shift is at least 64 when
// E >= 62; the column's scale then lies far below any value the tile can hold anyway).
__device__ __forceinline__ void digits52i(double x, int E, unsigned &hi, unsigned &lo) {
  const unsigned xh = (unsigned)__double2hiint(x), xl = (unsigned)__double2loint(x);
  const int e = (xh >> 20) & 0x7ff;
  const unsigned long long m = ((unsigned long long)((xh & 0xFFFFFu) | 0x100000u) << 32) | xl;
  const unsigned long long v = e ? m >> min(E + 2 - e, 63) : 0ull;
  const long long sv = ((int)xh < 0) ? -(long long)v : (long long)v;
  const unsigned long long w = (unsigned long long)sv + 0x0080808080808080ull;
  hi = (unsigned)(w >> 32);
  lo = (unsigned)w;
}
// two fp16 digits in one word: byte K (0 = least significant) of the values a (low half) and b
// (high half), each under the fp16 exponent of 1024, minus 1024 + 128 (exact)
template <int K>
__device__ __forceinline__ unsigned digit_pair(unsigned ahi, unsigned alo, unsigned bhi, unsigned blo) {
  constexpr unsigned k = K & 3;
  constexpr unsigned sel = k | (k << 4) | ((4 + k) << 8) | ((4 + k) << 12);
  const unsigned w = __byte_perm(K >= 4 ? ahi : alo, K >= 4 ? bhi : blo, sel);
  unsigned r;
  asm("{\n .reg .b32 t;\n lop3.b32 t, %1, %2, %3, 0xEA;\n sub.rn.f16x2 %0, t, %4;\n}\n"
      : "=r"(r) : "r"(w), "r"(0x00FF00FFu), "r"(0x64006400u), "r"(0x64806480u));
  return r;
}

}  // namespace

// One CTA: tiles blockIdx.x, blockIdx.x + gridDim.x, ... of the launch's virtual blocks (F_TCOLS
// numbering: per item, (Py - 2) middle rows x ceil(ncols / 64) column tiles, column tile fastest).
constexpr int TC_PREFETCH = 3;   // stages ahead of the L2 prefetch of the field

// ADJ: the adjoint's sums (k_adj_ring_cols) instead: A[r][q] = muhat(q, n) on the inner middle
// rows n = nlo + 2 + t, B at the ring columns mlo, mlo+1, mhi-1, mhi (the plan's second digit
// block), the 4 sums per row and column written to the workspace rows 2 Px + 4 t + s that
// k_adj_gamma reads, and with kind != 0 the k-gradient partials -Re <sum, s> of each warp of the
// first producer half, 4 per tile, into the item's reduction slots (summed in order by
// k_red_items).
template <bool CIN, bool ADJ>
__global__ void __launch_bounds__(TC_THREADS, 2)
    k_inv_cols_tc(Batch bt, const SubDesc *subs, const double *tab, const double *ws, const double2 *xi_user,
                  double2 *out, int kind, int *status) {
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  __shared__ __align__(8) unsigned long long full_bar[TC_STAGES], empty_bar[TC_STAGES], tfull_bar, tempty_bar, xbar;
  __shared__ unsigned tmem_slot;
  __shared__ double half_sh[128][5];        // the second producer half's 4 values per row (padded)
  __shared__ volatile int abort_sh;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full_bar[s])), "r"(TC_PRODUCERS) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty_bar[s])) : "memory");
    }
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tfull_bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&tempty_bar)), "r"(TC_PRODUCERS) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&xbar)), "r"(TC_PRODUCERS / 2) : "memory");
    abort_sh = 0;
  }
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TC_TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = tmem_slot;
  const unsigned sbase = smem_u32(tc_sm);

  if (warp == 8) {
    // ---------------------------------------------------------------- MMA warp
    if (lane == 0) {
      unsigned g = 0, T = 0;                  // stages and tiles processed (the barrier phases)
      for (int v = blockIdx.x; v < bt.total_blocks && !abort_sh; v += gridDim.x) {
        Item it; int local;
        locate(bt, v, it, local);
        if (MDP_CHECKED && !item_in_bounds(bt, subs, it, local, ADJ ? F_ATCOLS : F_TCOLS, ADJ)) continue;   // every warp skips it
        const int nchunk = (subs[it.sub].Nq + TC_KC - 1) / TC_KC;
        if (T > 0 && !mbar_wait(smem_u32(&tempty_bar), (T - 1) & 1u, &abort_sh)) break;
        tc_fence_after();
        bool ok = true;
        for (int c = 0; c < nchunk; ++c, ++g) {
          const unsigned st = g % TC_STAGES;
          if (!mbar_wait(smem_u32(&full_bar[st]), (g / TC_STAGES) & 1u, &abort_sh)) { ok = false; break; }
          tc_fence_after();
          const unsigned a0 = sbase + st * TC_STAGE_BYTES;
          const uint64_t db = smem_desc(a0 + TC_DIG * TC_A_BYTES, 128, 256);
          const unsigned acc = c > 0 ? 1u : 0u;
#pragma unroll
          for (int dgt = 0; dgt < TC_DIG; ++dgt) {
            const uint64_t da = smem_desc(a0 + dgt * TC_A_BYTES, 128, 256);
            asm volatile(
                "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + 32u * dgt),
                "l"(da), "l"(db), "r"(TC_IDESC), "r"(acc)
                : "memory");
          }
          tc_commit(smem_u32(&empty_bar[st]));
        }
        if (!ok) break;
        tc_commit(smem_u32(&tfull_bar));
        ++T;
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- producer warps
    const int quarter = warp & 3, half = warp >> 2;
    const int r = 32 * quarter + lane;        // matrix row of A (TMEM lane) of this thread
    unsigned g = 0, T = 0;                    // stages and tiles processed (the barrier phases)
    for (int v = blockIdx.x; v < bt.total_blocks && !abort_sh; v += gridDim.x) {
      Item it; int local;
      locate(bt, v, it, local);
      if (MDP_CHECKED && !item_in_bounds(bt, subs, it, local, ADJ ? F_ATCOLS : F_TCOLS, ADJ)) continue;     // every warp skips it
      const SubDesc &d = subs[it.sub];
      const bool CD = ADJ || d.cplx || CIN;
      const int nct = (it.ncols + 63) >> 6;
      const int t = local / nct, b0 = (local % nct) * 64;
      const int b = b0 + (r >> 1), ri = r & 1;
      const bool live = b < it.ncols && (CD || ri == 0);
      const int Nq = d.Nq;
      const int nchunk = (Nq + TC_KC - 1) / TC_KC;
      int rbase[5];
      if (ADJ) red_slots(d, it.ncols, rbase);
      // this thread's value of mode q = 1 at y, of mode q at y + (q - 1) qstride; the column's
      // scale: its largest biased exponent, recorded by the sweep that stored the field
      const double *y;
      long long qstride;
      int E;
      if (ADJ) {
        const int j = d.nlo + 2 + t - d.nfirst;   // inner middle row n = nlo + 2 + t (matrix numbering)
        qstride = 2LL * d.Nt * it.ncols;
        y = ws + it.a_off + 2LL * ((long long)j * it.ncols + b) + ri;
        E = live ? reinterpret_cast<const int *>(ws + it.red_off + rbase[4] + 1)[b] : 0;
      } else {
        const int yrow = t + 2;                 // middle row n = nlo + 1 + t
        const long long ncd = (long long)it.ncols * (CD ? 2 : 1);   // doubles per stored row
        qstride = (long long)d.NYf * ncd;
        y = ws + it.y_off + (long long)yrow * ncd + (CD ? 2LL * b + ri : (long long)b);
        E = live ? reinterpret_cast<const int *>(ws + it.red_off)[b] : 0;
      }
      const long long mb = magic_bits(E);
      const double magic = __longlong_as_double(mb);
      const long long cb = mb - 0x0080808080808080LL;
      // this thread's 8 modes of a stage: the current ones in xv, the next ones in flight in xn
      double xv[8], xn[8];
      auto load8 = [&](double *dst, int c) {
        const int q0 = c * TC_KC + 1 + 8 * half;
        const double *p = y + (long long)(q0 - 1) * qstride;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          dst[j] = (live && q0 + j <= Nq) ? *p : 0.0;
          p += qstride;
        }
      };
      // the values TC_PREFETCH stages ahead are prefetched into L2 (no registers held), so the
      // register loads one stage ahead find them there
      auto prefetch8 = [&](int c) {
        const int q0 = c * TC_KC + 1 + 8 * half;
        const double *p = y + (long long)(q0 - 1) * qstride;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (live && q0 + j <= Nq) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
          p += qstride;
        }
      };
      for (int c = 1; c < TC_PREFETCH && c < nchunk; ++c) prefetch8(c);
      load8(xv, 0);
      bool ok = true;
      for (int c = 0; c < nchunk; ++c, ++g) {
        if (c + TC_PREFETCH < nchunk) prefetch8(c + TC_PREFETCH);
        if (c + 1 < nchunk) load8(xn, c + 1);
        const unsigned st = g % TC_STAGES;
        // the stage is free once the MMAs that last read it have completed
        if (g >= TC_STAGES && !mbar_wait(smem_u32(&empty_bar[st]), (g / TC_STAGES - 1) & 1u, &abort_sh)) {
          ok = false;
          break;
        }
        unsigned char *sa = tc_sm + st * TC_STAGE_BYTES;
        {
          unsigned hi[8], lo[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            // the FP64 add takes half the values, the integer pipes the other half: each alone
            // would bound the stage
            if (j & 1) digits52i(xv[j], E, hi[j], lo[j]);
            else digits52(xv[j], magic, cb, hi[j], lo[j]);
          }
          const int off = (r >> 3) * 256 + half * 128 + (r & 7) * 16;   // SBO 256 B, LBO 128 B
#define MDP_TC_DIGIT(T)                                                                                     \
  {                                                                                                         \
    uint4 w;                                                                                                \
    w.x = digit_pair<6 - (T)>(hi[0], lo[0], hi[1], lo[1]);                                                 \
    w.y = digit_pair<6 - (T)>(hi[2], lo[2], hi[3], lo[3]);                                                 \
    w.z = digit_pair<6 - (T)>(hi[4], lo[4], hi[5], lo[5]);                                                 \
    w.w = digit_pair<6 - (T)>(hi[6], lo[6], hi[7], lo[7]);                                                 \
    *reinterpret_cast<uint4 *>(sa + (T) * TC_A_BYTES + off) = w;                                            \
  }
          MDP_TC_DIGIT(0) MDP_TC_DIGIT(1) MDP_TC_DIGIT(2) MDP_TC_DIGIT(3) MDP_TC_DIGIT(4) MDP_TC_DIGIT(5)
          MDP_TC_DIGIT(6)
#undef MDP_TC_DIGIT
        }
        // B: the plan's 1 KiB block of sine digits for these 16 modes, 16 bytes per thread
        if (tid < 64)
          *reinterpret_cast<uint4 *>(sa + TC_DIG * TC_A_BYTES + 16 * tid) =
              reinterpret_cast<const uint4 *>(tab + d.tcb_off + (ADJ ? 128LL * nchunk : 0LL))[c * 64 + tid];
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic stores -> MMA reads
        mbar_arrive(smem_u32(&full_bar[st]));
#pragma unroll
        for (int j = 0; j < 8; ++j) xv[j] = xn[j];
      }
      if (!ok) break;
      // ---- epilogue: D_t[r][8 so + u] = sum_q A_t B_u. x = V 2^(E - 1073), sin = W 2^-50, so the
      // weight of (t, u) is 2^(E - 1123 + 8 (12 - t - u)) = 2^(E - 1027 - 8 (t + u))
      if (!mbar_wait(smem_u32(&tfull_bar), T & 1u, &abort_sh)) break;
      tc_fence_after();
      // products of weight c = t + u, as integers: P0 = sum_{c<=3} I_c 2^(8 (3 - c)),
      // P1 = sum_{4<=c<=7} I_c 2^(8 (7 - c)), P2 = sum_{c>=8} I_c 2^(8 (12 - c)) (all below 2^60)
      auto pow2 = [](int k) { return k < -1022 ? 0.0 : __longlong_as_double((long long)(k + 1023) << 52); };
      const int Ec = min(max(E, 0), 2044);
      const double s0 = pow2(Ec - 1051), s1 = pow2(Ec - 1083), s2 = pow2(Ec - 1123), sc = 2.0 / d.Nx;
      long long acc[4][3];
#pragma unroll
      for (int so = 0; so < 4; ++so) acc[so][0] = acc[so][1] = acc[so][2] = 0;
      // this warp's A digits: 0..3 (first half) or 4..6 (second half), one load and wait each
#pragma unroll
      for (int ta = 0; ta < TC_DIG; ++ta) {
        if ((ta < 4) != (half == 0)) continue;
        float dv[32];
        tmem_ld32(tmem + ((unsigned)(32 * quarter) << 16) + 32u * ta, dv);
#pragma unroll
        for (int so = 0; so < 4; ++so)
#pragma unroll
          for (int u = 0; u < TC_DIG; ++u) {
            const int cw = ta + u;
            const long long iv = (long long)__float2int_rn(dv[so * 8 + u]);
            if (cw <= 3) acc[so][0] += iv * (1LL << (8 * (3 - cw)));
            else if (cw <= 7) acc[so][1] += iv * (1LL << (8 * (7 - cw)));
            else acc[so][2] += iv * (1LL << (8 * (12 - cw)));
          }
      }
      double val[4];
#pragma unroll
      for (int so = 0; so < 4; ++so)
        val[so] = sc * fma((double)acc[so][0], s0, fma((double)acc[so][1], s1, (double)acc[so][2] * s2));
      tc_fence_before();
      mbar_arrive(smem_u32(&tempty_bar));     // D may be overwritten by the next tile
      if (half == 1) {
        for (int so = 0; so < 4; ++so) half_sh[r][so] = val[so];
        mbar_arrive(smem_u32(&xbar));         // (release: the values above are visible to the waiters)
      } else {
        if (!mbar_wait(smem_u32(&xbar), T & 1u, &abort_sh)) break;
        for (int so = 0; so < 4; ++so) val[so] += half_sh[r][so];
        double u4[4];
        if (d.xsym) {
          u4[0] = val[0] + val[2]; u4[1] = val[1] + val[3]; u4[2] = val[1] - val[3]; u4[3] = val[0] - val[2];
        } else {
          u4[0] = val[0]; u4[1] = val[1]; u4[2] = val[2]; u4[3] = val[3];
        }
        if (ADJ) {
          // each lane writes its part (real: even lane, imaginary: odd lane) of the 4 sums
          double *wsw = const_cast<double *>(ws);   // rows and slots no other lane of the launch reads
          double part = 0.0;
          if (b < it.ncols) {
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              const long long o = 2LL * ((long long)(2 * d.Px + 4 * t + s) * it.ncols + b) + ri;
              wsw[it.r_off + o] = u4[s];
              if (kind) part = fma(-u4[s], ws[it.s_off + o], part);
            }
          }
          if (kind) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
            if (lane == 0) wsw[it.red_off + rbase[2] + 4 * local + quarter] = part;
          }
        } else {
          // lanes 2i (real part) and 2i+1 (imaginary part) of column b: the even lane writes
          double o4[4];
#pragma unroll
          for (int s = 0; s < 4; ++s) o4[s] = __shfl_xor_sync(0xffffffffu, u4[s], 1);
          if (ri == 0 && b < it.ncols) {
            const int g0 = 2 * (d.Px + 2) + 4 * t;
#pragma unroll
            for (int s = 0; s < 4; ++s) {
              cplx uv = cmk(-u4[s], CD ? -o4[s] : 0.0);
              if (kind == MDP_OUT_P) uv = cadd(uv, density<CIN>(d, it, ws, tab, xi_user, b, g0 + s));
              out[it.io_off + (long long)b * d.G + g0 + s] = make_double2(uv.re, uv.im);
            }
          }
        }
      }
      // half_sh is rewritten only in the next tile's epilogue, which no producer reaches before
      // every producer has filled that tile's stages (and so finished reading here)
      ++T;
    }
  }
  if (abort_sh && tid == 0) atomicCAS(status, 0, (int)MDP_ERR_TIMEOUT);   // the first error sticks
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

int tc_cols_smem_bytes() { return TC_STAGES * TC_STAGE_BYTES; }

cudaError_t set_tc_kernel_attributes() {
  const int sm = tc_cols_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(k_inv_cols_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_cols_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_inv_cols_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  return e;
}

cudaError_t launch_inv_cols_tc(const Batch &b, const SubDesc *subs, const double *tab, const double *ws,
                               const double2 *xi_user, double2 *out, int kind, int *status, int n_sm,
                               cudaStream_t st) {
  const int grid = std::max(1, std::min(b.total_blocks, 2 * n_sm));
  if (xi_user)
    k_inv_cols_tc<true, false><<<grid, TC_THREADS, tc_cols_smem_bytes(), st>>>(b, subs, tab, ws, xi_user, out, kind, status);
  else
    k_inv_cols_tc<false, false><<<grid, TC_THREADS, tc_cols_smem_bytes(), st>>>(b, subs, tab, ws, xi_user, out, kind, status);
  return cudaGetLastError();
}

cudaError_t launch_adj_cols_tc(const Batch &b, const SubDesc *subs, const double *tab, double *ws, bool dk,
                               int *status, int n_sm, cudaStream_t st) {
  const int grid = std::max(1, std::min(b.total_blocks, 2 * n_sm));
  k_inv_cols_tc<false, true><<<grid, TC_THREADS, tc_cols_smem_bytes(), st>>>(b, subs, tab, ws, nullptr, nullptr,
                                                                            dk ? 1 : 0, status);
  return cudaGetLastError();
}

}  // namespace mdp
