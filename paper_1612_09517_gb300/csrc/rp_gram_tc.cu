// The exact time integral of a macro-step (Eqs. 20, 22) on the tensor cores:
// tcgen05.mma kind::tf32 on hi/lo-split FP32 singlet slices, accumulators in
// tensor memory drained into FP32 partial sums in registers, FP64 contraction
// with the time-integral weights.
#include <stdint.h>

#include "rp_device.cuh"
#include "rp_kernels.cuh"

namespace rp {

namespace {

// ---- Exact time integral on the tensor cores (FP32 state, tcgen05 3xTF32) ----
//
// The same quantity as k_gram_integrate (Eqs. 20, 22): integral[r] +=
// Re sum_nm W_nm G_nm with G_nm = sum_z conj(x_n(z)) x_m(z).  With the real
// rows a = 2n + p (p = 0: Re x_n, p = 1: Im x_n) of the singlet slices as a
// (2 n_c) x Z matrix A, the real Gram R = A A^T holds G (Re G_nm = R_{2n,2m} +
// R_{2n+1,2m+1}, Im G_nm = R_{2n,2m+1} - R_{2n+1,2m}), and the integral is
// sum_ab What_ab R_ab with the symmetric What_{2n+p,2m+q} = Re W_nm (p = q),
// -Im W_nm (p = 0, q = 1), Im W_nm (p = 1, q = 0).
//
// One CTA (512 threads, one per SM) takes a range of kXChunk-configuration
// chunks of one row.  Per chunk: one bulk copy (the chunk is contiguous in the
// layout written by the step kernel) into a stage of a kGramStages-deep ring
// on mbarriers; the threads split each value into hi = its nearest TF32 and
// lo = the nearest TF32 of value - hi; one thread issues tcgen05.mma
// kind::tf32 for hi.hi + hi.lo + lo.hi into FP32 accumulators in tensor
// memory: D1 = A[0:128] A[0:R2p]^T (128 x R2p) and, when 2 n_c > 128,
// D2 = A[R2p-128:R2p] A[128:R2p]^T, the lower-right block (R2p = 2 n_c
// rounded up to 16).  The product of two split values misses lo.lo and the
// rounding of lo: at most about 2^-21 of |x_n x_m|, unbiased except lo.lo on
// the diagonal (about 2^-24).
//
// The tensor core's FP32 accumulation is not round-to-nearest: its error grows
// with the number of MMAs added into one accumulator and has one sign.  So
// every kGramGroup chunks (12 MMAs per accumulator) the accumulator buffer is
// drained with tcgen05.ld into FP32 partial sums held in registers
// (round-to-nearest adds), while the tensor core fills the other buffer.  Each
// thread owns one accumulator row (its warp's tensor-memory lane quarter) and
// a quarter of the columns.  At the end the partial sums are contracted with
// What in FP64 (entries of D1 with column >= 128 twice: R is symmetric and D2
// holds only the lower-right block) and the CTA adds one FP64 atomic.  Every
// wait is bounded; a wait that gives up sets bit 0 of the error word, lets
// the copies and MMAs in flight land, frees tensor memory and returns.
constexpr int kGramStages = 6;  // a multiple of kGramGroup
constexpr int kGramCpgMax = 56;  // partial-sum columns per thread (n_c <= 88)
constexpr int kGramGroup = 2;  // chunks accumulated in tensor memory before a drain
static_assert(kGramStages % kGramGroup == 0, "stages hold whole groups");
constexpr int kGramTcThreads = 512;  // 16 warps: 4 per tensor-memory lane quarter
constexpr int kGramTmemCols = 512;  // two accumulator buffers, 256 columns apart
constexpr int kGramMinSmem = 116 * 1024;  // keeps one CTA (and 512 TMEM columns) per SM
constexpr long long kWaitLimit = 1ll << 24;

__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (long long it = 0; it < kWaitLimit; ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes,
                                          unsigned bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// tcgen05 shared-memory matrix descriptor, K-major, no swizzle: start address,
// leading byte offset (next core matrix along K), stride byte offset (next
// 8-row group), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(unsigned addr, unsigned lbo, unsigned sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(unsigned d, uint64_t a, uint64_t b, uint32_t idesc,
                                         unsigned accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(unsigned bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void tmem_ld4(unsigned taddr, float (&v)[4]) {
  uint32_t u[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float (&v)[8]) {
  uint32_t u[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]),
                 "=r"(u[6]), "=r"(u[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(u[i]);
}

__device__ __forceinline__ void tmem_ld16(unsigned taddr, float (&v)[16]) {
  uint32_t u[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(u[0]), "=r"(u[1]), "=r"(u[2]), "=r"(u[3]), "=r"(u[4]), "=r"(u[5]), "=r"(u[6]),
        "=r"(u[7]), "=r"(u[8]), "=r"(u[9]), "=r"(u[10]), "=r"(u[11]), "=r"(u[12]), "=r"(u[13]),
        "=r"(u[14]), "=r"(u[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(u[i]);
}

// Nearest TF32 value of a finite float (ties away from zero): add half a unit
// of the 10-bit mantissa and clear the 13 low bits.  hi and lo are both exact
// TF32 numbers, so the tensor core uses them unchanged and the split errors
// are unbiased rounding errors.
__device__ __forceinline__ float tf32_round(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// What_{a j} for the row-pair interleaved real Gram (see above).
__device__ __forceinline__ double what(const double* __restrict__ Wf, int n_c, int a, int j) {
  const int n = a >> 1, m = j >> 1;
  const double* w = Wf + ((size_t)n * n_c + m) * 2;
  if ((a & 1) == (j & 1)) return w[0];
  return (a & 1) ? w[1] : -w[1];
}

__global__ void __launch_bounds__(kGramTcThreads, 1) k_gram_tc(
    const float* __restrict__ X, const double* __restrict__ W, const int* __restrict__ row_field,
    const int2* __restrict__ row_win, int macro_arg, const int* __restrict__ macro_dev, int n_c,
    long long Zs, const HamDev<float>* __restrict__ ham, const int* __restrict__ row_sys,
    int chunks_per_cta, double* __restrict__ integral, int* __restrict__ err) {
  const int r = blockIdx.y;
  {
    const int macro = macro_dev ? *macro_dev : macro_arg;
    const int2 w = row_win[r];
    if (macro < w.x || macro >= w.y) return;
  }
  // chunks of this row's own system (rows of one launch may differ in Z)
  const long long Zr = ham[row_sys ? row_sys[r] : 0].Z;
  const int n_chunks = (int)((Zr + kXChunk - 1) / kXChunk);
  const int c_begin = blockIdx.x * chunks_per_cta;
  const int nk = min(n_chunks - c_begin, chunks_per_cta);
  if (nk <= 0) return;
  const int R2 = 2 * n_c, R2p = xrows_pad(n_c);
  const int N1 = R2p, N2 = R2p > 128 ? R2p - 128 : 0, NT = N1 + N2;
  const unsigned copy_bytes = (unsigned)R2p * kXChunk * 4;
  const unsigned tile_bytes = (unsigned)(R2p > 128 ? R2p : 128) * kXChunk * 4;

  extern __shared__ __align__(1024) unsigned char gram_smem[];
  // barriers: full[stage], empty[stage], acc_ready[buffer], fin (error path)
  __shared__ __align__(8) unsigned long long bars[2 * kGramStages + 3];
  __shared__ unsigned tmem_slot;
  __shared__ double red[kGramTcThreads];
  const unsigned tid = threadIdx.x, warp = tid >> 5;
  const unsigned sbase = smem_u32(gram_smem);
  auto hi_tile = [&](int s) { return sbase + (unsigned)(2 * s) * tile_bytes; };
  auto lo_tile = [&](int s) { return sbase + (unsigned)(2 * s + 1) * tile_bytes; };
  auto full = [&](int s) { return smem_u32(&bars[s]); };
  auto empty = [&](int s) { return smem_u32(&bars[kGramStages + s]); };
  auto ready = [&](int b) { return smem_u32(&bars[2 * kGramStages + b]); };
  // FP32 partial sums of this CTA's Gram rows, in registers: thread (warp w,
  // lane l) owns row a = 32 (w % 4) + l (the tensor-memory lanes its warp may
  // read) and columns j0 .. j0 + cpg - 1, the column group w / 4 of NT / 4.
  const int a_row = (int)((warp & 3u) * 32u + (tid & 31u));
  const int cpg = NT / 4, j0 = (int)(warp >> 2) * cpg;
  float accr[kGramCpgMax];
#pragma unroll
  for (int i = 0; i < kGramCpgMax; ++i) accr[i] = 0.f;

  if (tid == 0) {
    for (int i = 0; i < 2 * kGramStages + 3; ++i)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&bars[i])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kGramTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const unsigned tmem = tmem_slot;
  const unsigned lane_base = tmem + (((warp & 3u) * 32u) << 16);

  const float* src = X + (size_t)r * xblk_row_floats(Zs, n_c) + (size_t)c_begin * R2p * kXChunk;
  int issued = 0;
  if (tid == 0) {
    for (; issued < nk && issued < kGramStages; ++issued)
      bulk_load(hi_tile(issued), src + (size_t)issued * R2p * kXChunk, copy_bytes, full(issued));
  }
  const uint32_t id1 = idesc_tf32(128, N1), id2 = idesc_tf32(128, N2 > 0 ? N2 : 16);
  int failed = 0;  // this thread saw a wait give up
  int consumed = 0;
  // adds accumulator buffer gg % 2 (group gg) into acc, all threads
  // (the tensor-memory loads are warp-collective, so they run even after a
  // failed wait; the CTA then discards its sum)
  auto drain = [&](int gg) {
    if (!mbar_wait(ready(gg & 1), (unsigned)(gg >> 1) & 1u)) failed = 1;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned col0 = (unsigned)(gg & 1) * 256u + (unsigned)j0;
    if (cpg % 8 == 0) {
#pragma unroll
      for (int i = 0; i < kGramCpgMax / 8; ++i) {
        if (8 * i < cpg) {  // the same for the whole warp
          float v[8];
          tmem_ld8(lane_base + col0 + 8u * i, v);
#pragma unroll
          for (int t = 0; t < 8; ++t) accr[8 * i + t] += v[t];
        }
      }
    } else {
#pragma unroll
      for (int i = 0; i < kGramCpgMax / 4; ++i) {
        if (4 * i < cpg) {
          float v[4];
          tmem_ld4(lane_base + col0 + 4u * i, v);
#pragma unroll
          for (int t = 0; t < 4; ++t) accr[4 * i + t] += v[t];
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  };
  const int n_groups = (nk + kGramGroup - 1) / kGramGroup;
  // one block barrier per group of kGramGroup chunks (kGramStages is a multiple)
  for (int g = 0; g < n_groups; ++g) {
    const int k0 = g * kGramGroup, k1 = min(nk, k0 + kGramGroup);
    for (int kc = k0; kc < k1; ++kc) {
      const int s = kc % kGramStages;
      if (!mbar_wait(full(s), (unsigned)(kc / kGramStages) & 1u)) {
        failed = 1;
        continue;
      }
      float4* h = reinterpret_cast<float4*>(gram_smem + (size_t)(2 * s) * tile_bytes);
      float4* l = reinterpret_cast<float4*>(gram_smem + (size_t)(2 * s + 1) * tile_bytes);
      for (int q = (int)tid; q < R2p * kXChunk / 4; q += kGramTcThreads) {
        const float4 v = h[q];
        const float4 hv = make_float4(tf32_round(v.x), tf32_round(v.y), tf32_round(v.z),
                                      tf32_round(v.w));
        h[q] = hv;
        l[q] = make_float4(tf32_round(v.x - hv.x), tf32_round(v.y - hv.y), tf32_round(v.z - hv.z),
                           tf32_round(v.w - hv.w));
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (__syncthreads_or(failed)) break;
    consumed = k1;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const unsigned dbase = tmem + (unsigned)(g & 1) * 256u;
      for (int kc = k0; kc < k1; ++kc) {
        const int s = kc % kGramStages;
        const unsigned A[3] = {hi_tile(s), hi_tile(s), lo_tile(s)};
        const unsigned B[3] = {hi_tile(s), lo_tile(s), hi_tile(s)};
#pragma unroll
        for (int ks = 0; ks < kXChunk / 8; ++ks)
#pragma unroll
          for (int pr = 0; pr < 3; ++pr) {
            const unsigned accumulate = (kc > k0 || ks > 0 || pr > 0) ? 1u : 0u;
            const unsigned ko = (unsigned)ks * 256;  // two core matrices of 4 configurations
            mma_tf32(dbase, umma_desc(A[pr] + ko, 128, 512), umma_desc(B[pr] + ko, 128, 512),
                     id1, accumulate);
            if (N2 > 0)
              mma_tf32(dbase + (unsigned)N1,
                       umma_desc(A[pr] + (unsigned)((R2p - 128) / 8) * 512 + ko, 128, 512),
                       umma_desc(B[pr] + 16u * 512 + ko, 128, 512), id2, accumulate);
          }
        mma_commit(empty(s));
      }
      mma_commit(ready(g & 1));
      // refill the stages of the previous group once its MMAs are done
      for (int kp = k0 - kGramGroup; kp >= 0 && kp < k0; ++kp) {
        const int nxt = kp + kGramStages;
        if (nxt >= nk) break;
        const int sp = kp % kGramStages;
        if (mbar_wait(empty(sp), (unsigned)(kp / kGramStages) & 1u)) {
          bulk_load(hi_tile(sp), src + (size_t)nxt * R2p * kXChunk, copy_bytes, full(sp));
          ++issued;
        } else {
          failed = 1;
          break;
        }
      }
    }
    // the previous group's buffer drains while the tensor core works on this one
    if (g >= 1) drain(g - 1);
  }
  const bool completed = consumed == nk;
  if (__syncthreads_or(failed) == 0 && completed) drain(n_groups - 1);
  const int bad = __syncthreads_or(failed || !completed);
  double sum = 0.0;
  if (!bad) {
    const double* Wf = W + (size_t)row_field[r] * n_c * n_c * 2;
    const int a = a_row, a2 = R2p - 128 + a_row;
#pragma unroll
    for (int i = 0; i < kGramCpgMax; ++i) {
      const int j = j0 + i;
      if (i >= cpg) break;
      if (j < N1) {  // D1 entry (a, j); columns >= 128 stand for their transposes too
        if (a < R2 && j < R2)
          sum += (j >= 128 ? 2.0 : 1.0) * what(Wf, n_c, a, j) * (double)accr[i];
      } else {  // D2 entry (a2, 128 + j - N1) of the lower-right block
        const int jj = 128 + j - N1;
        if (a2 >= 128 && a2 < R2 && jj < R2) sum += what(Wf, n_c, a2, jj) * (double)accr[i];
      }
    }
  } else {
    if (tid == 0) {
      if (err) atomicOr(err, 1);
      // copies issued but not consumed still land in shared memory; MMAs issued
      // still run: wait for both before the tensor memory is freed
      for (int c = consumed; c < issued; ++c)
        mbar_wait(full(c % kGramStages), (unsigned)(c / kGramStages) & 1u);
      const unsigned fin = smem_u32(&bars[2 * kGramStages + 2]);
      mma_commit(fin);  // arrives once every MMA issued so far has completed
      mbar_wait(fin, 0);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kGramTmemCols)
                 : "memory");
  if (!bad) {
    const double tot = block_sum<kGramTcThreads>(sum, red);
    if (tid == 0) atomicAdd(integral + r, tot);
  }
}

}  // namespace

size_t gram_tc_smem_bytes(int n_c) {
  const int R2p = xrows_pad(n_c);
  const size_t b = (size_t)2 * kGramStages * (R2p > 128 ? R2p : 128) * kXChunk * 4;
  return b > (size_t)kGramMinSmem ? b : (size_t)kGramMinSmem;
}

size_t smem_max_gram_tc() { return gram_tc_smem_bytes(88); }

// both accumulator blocks (2 R2p - 128 columns) fit one 256-column buffer and
// a quarter of them fits the per-thread partial sums (kGramCpgMax)
bool gram_tc_supported(int n_c) { return n_c >= 8 && n_c <= 88; }

cudaError_t launch_gram_tc(const float* X, const double* W, const int* row_field,
                           const int2* row_win, int macro, const int* macro_dev, int rows, int n_c,
                           long long Zs, const HamDev<float>* ham, const int* row_sys, int n_sm,
                           double* integral, int* err, cudaStream_t st) {
  if (rows == 0) return cudaSuccess;
  if (!gram_tc_supported(n_c)) return cudaErrorInvalidValue;
  const size_t smem = gram_tc_smem_bytes(n_c);
  static std::atomic<unsigned long long> attr_done;
  const cudaError_t ea = smem_attr_once((const void*)k_gram_tc, (int)smem_max_gram_tc(), attr_done);
  if (ea != cudaSuccess) return ea;
  // chunks per CTA: the split of each row that minimises (waves of resident
  // CTAs) x (chunks per CTA + a fixed cost for fill and epilogue)
  const long long n_chunks = (Zs + kXChunk - 1) / kXChunk;
  const long long resident = n_sm > 0 ? n_sm : 1;  // one CTA per SM (shared memory)
  long long per = n_chunks, best = -1;
  for (long long cpr = 1; cpr <= 256 && cpr <= n_chunks; ++cpr) {
    const long long p = (n_chunks + cpr - 1) / cpr;
    const long long ctas = (long long)rows * ((n_chunks + p - 1) / p);
    const long long cost = ((ctas + resident - 1) / resident) * (p + 24);
    if (best < 0 || cost < best) {
      best = cost;
      per = p;
    }
  }
  dim3 grid((unsigned)((n_chunks + per - 1) / per), rows);
  k_gram_tc<<<grid, kGramTcThreads, smem, st>>>(X, W, row_field, row_win, macro, macro_dev, n_c, Zs,
                                                ham, row_sys, (int)per, integral, err);
  return cudaGetLastError();
}

}  // namespace rp
