// X = Z Y on the tensor cores (see assemble_tc.cuh for the slicing scheme).
//
// Kernels: k_tc_slice_a (row exponents and slices of [Re z, Im z]),
// k_tc_slice_b (column exponents and slices of the interleaved Y columns) and
// k_tc_gemm: one CTA per (32-column tile, 128-row tile, source); one thread
// streams 16-wide k' slabs of all slices into shared memory with bulk async
// copies (two stages, mbarrier transaction counts) and issues the 36
// tcgen05.mma per slab into eight TMEM accumulators; after each chunk of at
// most 8 slabs four warps read the accumulators with tcgen05.ld into 64-bit
// totals (the copies of the next chunk's first slab already in flight), and
// after the last chunk write x_j. Every wait on an mbarrier gives up after two
// seconds, sets the error flag and still releases TMEM.
#include <algorithm>

#include "assemble_tc.cuh"

namespace fks {

namespace {

constexpr int STAGE_BYTES = TC_A_SLAB + TC_B_SLAB;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  uint64_t t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((it & 63) == 0) {
      uint64_t t = global_ns();
      if (t0 == 0) t0 = t;
      else if (t - t0 > 2000000000ull) return false;
    }
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: no swizzle, K-major core matrices of 8 rows x
// 16 bytes; lbo = byte step between the two core matrices along k, sbo = byte
// step between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100 and later
  return d;                // base offset 0, relative lbo, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::f16: bf16 A and B (K-major), fp32 D, M = 128,
// N columns (a multiple of 16, at most 256).
__host__ __device__ constexpr uint32_t mma_idesc(uint32_t N) {
  return (1u << 4)                        // D format: f32
         | (1u << 7)                      // A format: bf16
         | (1u << 10)                     // B format: bf16
         | ((N >> 3) << 17)               // N / 8
         | ((uint32_t)(TC_M >> 4) << 24); // M / 16
}

__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

// eight columns of the warp's 32 TMEM lanes; the values may be used only after tmem_wait
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Sources whose step count keeps the padded 2K within the exactness bound.
__host__ __device__ __forceinline__ bool tc_slot(int K) {
  return K >= 0 && ((2 * K + TC_KSLAB - 1) / TC_KSLAB) * TC_KSLAB <= TC_MAX_KP;
}

// Exponent e with max |row| < 2^e (0 for a zero row): for a normal amax, its
// biased exponent - 1022 (as frexp gives), read from the bits.
__device__ __forceinline__ int pow2_above(double amax) {
  if (amax == 0.0) return 0;
  const int be = (int)((__double_as_longlong(amax) >> 52) & 0x7FF);
  if (be != 0) return be - 1022;
  int e;
  frexp(amax, &e);  // subnormal
  return e;
}

// Eight signed 7-bit digits of v / 2^e (|v| < 2^e): v = 2^e sum_s d_s 2^{-7(s+1)}
// up to the truncated bits below 2^{e-56}. X = trunc(|v| 2^(56-e)) is the
// significand shifted by the exponent difference (integer instructions only).
__device__ __forceinline__ void digits7(double v, int e, int (&d)[TC_SLICES]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(v);
  const int be = (int)((bits >> 52) & 0x7FF);
  unsigned long long X;
  if (be == 0) {
    X = (unsigned long long)__double2ull_rz(scalbn(fabs(v), 56 - e));  // zero or subnormal
  } else {
    const unsigned long long M = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = be - 1019 - e;  // |v| = M 2^(be - 1075)
    X = sh >= 0 ? (M << sh) : (sh > -64 ? (M >> -sh) : 0ull);
  }
  const int sg = (bits >> 63) ? -1 : 1;
#pragma unroll
  for (int s = 0; s < TC_SLICES; ++s) d[s] = sg * (int)((X >> (49 - 7 * s)) & 127ull);
}

// (hi + lo 2^-28) 2^E rounded to the nearest double (ties to even), with integer
// instructions only: N = hi 2^28 + lo is exact in 128 bits (|hi| < 2^47), its
// leading 53 bits are rounded by the bits below them, and the exponent is set
// directly. Equal to scalbn(fma((double)lo, 0x1p-28, (double)hi), E) whenever
// the result is a normal double; returns false otherwise (the caller then takes
// that FP64 form).
__device__ __forceinline__ bool int_to_double(long long hi, long long lo, int E, double* out) {
  const __int128 N = ((__int128)hi << 28) + (__int128)lo;
  if (N == 0) {
    *out = 0.0;
    return true;
  }
  const unsigned long long sign = N < 0 ? 1ull : 0ull;
  const unsigned __int128 u = N < 0 ? (unsigned __int128)(-N) : (unsigned __int128)N;
  const unsigned long long uh = (unsigned long long)(u >> 64), ul = (unsigned long long)u;
  const int p = uh ? 127 - __clzll((long long)uh) : 63 - __clzll((long long)ul);  // leading bit
  unsigned long long m;
  int ex = p;
  if (p <= 52) {
    m = ul << (52 - p);
  } else {
    const int sh = p - 52;  // 1 .. 75
    const unsigned __int128 q = u >> sh;
    const unsigned __int128 rem = u - (q << sh), half = (unsigned __int128)1 << (sh - 1);
    m = (unsigned long long)q;
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m == (1ull << 53)) {
      m >>= 1;
      ++ex;
    }
  }
  const int be = ex + E - 28 + 1023;
  if (be < 1 || be > 2046) return false;
  *out = __longlong_as_double((long long)((sign << 63) | ((unsigned long long)be << 52) | (m & ((1ull << 52) - 1))));
  return true;
}

// bf16 bits of a small integer (exact: at most 8 significant bits)
__device__ __forceinline__ uint32_t bf16_of(int d) { return __float_as_uint((float)d) >> 16; }

__device__ __forceinline__ uint4 pack8(const int (&d)[8][TC_SLICES], int s) {
  uint4 w;
  w.x = bf16_of(d[0][s]) | (bf16_of(d[1][s]) << 16);
  w.y = bf16_of(d[2][s]) | (bf16_of(d[3][s]) << 16);
  w.z = bf16_of(d[4][s]) | (bf16_of(d[5][s]) << 16);
  w.w = bf16_of(d[6][s]) | (bf16_of(d[7][s]) << 16);
  return w;
}

}  // namespace

// Slices of A = [Re z_k, Im z_k] (k' = 2k, 2k + 1), one thread per row.
// Layout (16-byte rows): [slot][row tile][slab][slice][8-row group 16][k chunk 2][row 8].
__global__ void __launch_bounds__(TC_M) k_tc_slice_a(const SlotState* __restrict__ st, const z64* __restrict__ Z,
                                                      int64_t vsZ, int64_t n, int nslab, int nrt,
                                                      uint4* __restrict__ As, int* __restrict__ erow) {
  const int rt = blockIdx.x, slot = blockIdx.y, r = threadIdx.x;
  // this source's own steps: the columns of Z it wrote in this solve
  const int K = st[slot].k;
  if (!tc_slot(K)) return;
  const int64_t i = (int64_t)rt * TC_M + r;
  const z64* Zs = Z + slot * vsZ;
  double amax = 0.0;
  if (i < n)
    for (int k = 0; k < K; ++k) {
      z64 z = Zs[(int64_t)k * n + i];
      amax = fmax(amax, fmax(fabs(z.re), fabs(z.im)));
    }
  const int e = pow2_above(amax);
  erow[((int64_t)slot * nrt + rt) * TC_M + r] = e;
  const int g = r >> 3, rr = r & 7;
  uint4* base = As + (size_t)(slot * nrt + rt) * nslab * (TC_A_SLAB / 16);
  for (int c = 0; c < 2 * nslab; ++c) {
    int d[8][TC_SLICES];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = 4 * c + q;
      z64 z = (i < n && k < K) ? Zs[(int64_t)k * n + i] : mk(0.0, 0.0);
      digits7(z.re, e, d[2 * q]);
      digits7(z.im, e, d[2 * q + 1]);
    }
    const int slab = c >> 1, kc = c & 1;
    uint4* sb = base + (size_t)slab * (TC_A_SLAB / 16);
#pragma unroll
    for (int s = 0; s < TC_SLICES; ++s) sb[((s * 16 + g) * 2 + kc) * 8 + rr] = pack8(d, s);
  }
}

// Slices of B: column 2j = [Re y_j; -Im y_j], column 2j + 1 = [Im y_j; Re y_j],
// interleaved over k like A; y_{j,k} = 0 for k >= m_j. One thread per column.
// Layout: [slot][column tile][slab][slice][8-column group 4][k chunk 2][column 8].
__global__ void __launch_bounds__(TC_N) k_tc_slice_b(const SlotState* __restrict__ st, const z64* __restrict__ Y,
                                                      const int32_t* __restrict__ mj, int nf, int m, int nslab,
                                                      int nct, uint4* __restrict__ Bs, int* __restrict__ ecol) {
  const int ct = blockIdx.x, slot = blockIdx.y, c = threadIdx.x;
  const int K = st[slot].k;
  if (!tc_slot(K)) return;
  const int jp = ct * TC_N + c, j = jp >> 1, part = jp & 1;
  const int mjj = j < nf ? min((int)mj[(int64_t)slot * nf + j], K) : 0;
  const z64* y = Y + ((int64_t)slot * nf + (j < nf ? j : 0)) * m;
  auto val = [&](int kp) -> double {
    const int k = kp >> 1;
    if (k >= mjj) return 0.0;
    const z64 v = y[k];
    const int h = kp & 1;
    return part == 0 ? (h == 0 ? v.re : -v.im) : (h == 0 ? v.im : v.re);
  };
  double amax = 0.0;
  for (int kp = 0; kp < 2 * mjj; ++kp) amax = fmax(amax, fabs(val(kp)));
  const int e = pow2_above(amax);
  ecol[((int64_t)slot * nct + ct) * TC_N + c] = e;
  const int g = c >> 3, rr = c & 7;
  uint4* base = Bs + (size_t)(slot * nct + ct) * nslab * (TC_B_SLAB / 16);
  for (int cc = 0; cc < 2 * nslab; ++cc) {
    int d[8][TC_SLICES];
#pragma unroll
    for (int q = 0; q < 8; ++q) digits7(val(8 * cc + q), e, d[q]);
    const int slab = cc >> 1, kc = cc & 1;
    uint4* sb = base + (size_t)slab * (TC_B_SLAB / 16);
#pragma unroll
    for (int s = 0; s < TC_SLICES; ++s) sb[((s * 4 + g) * 2 + kc) * 8 + rr] = pack8(d, s);
  }
}

// Persistent form: one CTA per SM takes (source, 128-row tile) items in turn and
// runs every 32-column tile of an item. Warp P_EPI + 1 (one lane) issues the
// MMAs of a tile (per chunk of at most 8 slabs) into one of two TMEM
// accumulator sets, warp P_EPI (one lane) streams the slabs through a ring of
// PS stages, and the epilogue warps drain the other set into 64-bit totals and
// write x_j, so a tile's epilogue overlaps the next tile's MMAs: warp w reads
// TMEM lanes 32 (w mod 4) .. + 31 (one row per thread) and the EPI_COLS columns
// of group w / 4 of the tile, four warps per SM sub-partition to hide the
// latency of the integer epilogue. Barriers: full/empty per stage,
// tfull/tempty per accumulator set.
constexpr int PS = 4;
constexpr int P_EPI = 16;                  // epilogue warps
constexpr int EPI_COLS = TC_N * 4 / P_EPI; // columns of a tile per epilogue warp (8)
constexpr int P_THREADS = 32 * (P_EPI + 2);
constexpr uint32_t P_TMEM_COLS = 512;      // two sets of 8 levels x 32 columns

struct PBars {
  uint64_t full[PS], empty[PS], tfull[2], tempty[2], fin;
  uint32_t tslot;
  int abort;
};

constexpr int P_SMEM = PS * STAGE_BYTES + (int)sizeof(PBars) + 64;

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ bool p_aborted(const PBars* B) { return *(volatile const int*)&B->abort != 0; }

__device__ __forceinline__ void p_fail(PBars* B, int* err, int code) {
  atomicExch(err, code);
  atomicExch(&B->abort, 1);
}

__global__ void __launch_bounds__(P_THREADS, 1) k_tc_gemm(const SlotState* __restrict__ st,
                                                           const unsigned char* __restrict__ As,
                                                           const unsigned char* __restrict__ Bs,
                                                           const int* __restrict__ erow, const int* __restrict__ ecol,
                                                           int nslab, int nrt, int nct, int64_t n, int nf, int nslot,
                                                           z64* __restrict__ X, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  PBars* B = reinterpret_cast<PBars*>(sm + PS * STAGE_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = smem_u32(sm);
  if (threadIdx.x == 0) {
    for (int q = 0; q < PS; ++q) {
      mbar_init(smem_u32(&B->full[q]), 1);
      mbar_init(smem_u32(&B->empty[q]), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(smem_u32(&B->tfull[a]), 1);
      mbar_init(smem_u32(&B->tempty[a]), P_EPI);
    }
    mbar_init(smem_u32(&B->fin), 1);
    B->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&B->tslot)),
                 "r"(P_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = B->tslot;
  constexpr int SPC = TC_CHUNK_KP / TC_KSLAB;  // slabs per chunk
  const int nchunk = (nslab + SPC - 1) / SPC;
  const int nitems = nslot * nrt;

  if (warp == P_EPI) {
    // ---- producer: slabs of every tile of every item, in order, through the ring
    if (lane == 0) {
      long long g = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x) {
        const int slot = item / nrt, rt = item - slot * nrt;
        if (!tc_slot(st[slot].k)) continue;
        const unsigned char* asrc = As + (size_t)(slot * nrt + rt) * nslab * TC_A_SLAB;
        for (int ct = 0; ok && ct < nct; ++ct) {
          const unsigned char* bsrc = Bs + (size_t)(slot * nct + ct) * nslab * TC_B_SLAB;
          for (int q = 0; q < nslab; ++q, ++g) {
            const int sg = (int)(g % PS);
            if (g >= PS && !mbar_wait(smem_u32(&B->empty[sg]), (uint32_t)((g / PS - 1) & 1))) {
              p_fail(B, err, 1);
              ok = false;
              break;
            }
            if (p_aborted(B)) { ok = false; break; }
            const uint32_t dst = sbase + sg * STAGE_BYTES, fb = smem_u32(&B->full[sg]);
            mbar_expect_tx(fb, STAGE_BYTES);
            bulk_g2s(dst, asrc + (size_t)q * TC_A_SLAB, TC_A_SLAB, fb);
            bulk_g2s(dst + TC_A_SLAB, bsrc + (size_t)q * TC_B_SLAB, TC_B_SLAB, fb);
          }
        }
      }
      // the copies of the last slabs must have landed before the CTA exits
      for (long long h = g - 1; h >= 0 && h >= g - PS; --h)
        mbar_wait(smem_u32(&B->full[h % PS]), (uint32_t)((h / PS) & 1));
    }
  } else if (warp == P_EPI + 1) {
    // ---- MMA issuer
    if (lane == 0) {
      long long g = 0;
      int u = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x) {
        const int slot = item / nrt;
        if (!tc_slot(st[slot].k)) continue;
        for (int ct = 0; ok && ct < nct; ++ct)
          for (int ch = 0; ok && ch < nchunk; ++ch, ++u) {
            const int acc = u & 1;
            if (u >= 2 && !mbar_wait(smem_u32(&B->tempty[acc]), (uint32_t)(((u >> 1) - 1) & 1))) {
              p_fail(B, err, 2);
              ok = false;
              break;
            }
            if (p_aborted(B)) { ok = false; break; }
            tc_fence_after();
            const uint32_t dacc = tmem + (uint32_t)(acc * 8 * TC_N);
            const int q1 = min(nslab, (ch + 1) * SPC);
            for (int q = ch * SPC; q < q1; ++q, ++g) {
              const int sg = (int)(g % PS);
              if (!mbar_wait(smem_u32(&B->full[sg]), (uint32_t)((g / PS) & 1))) {
                p_fail(B, err, 3);
                ok = false;
                break;
              }
              tc_fence_after();
              const uint32_t a0 = sbase + sg * STAGE_BYTES, b0 = a0 + TC_A_SLAB;
              // slice s of A times B slices t = 0 .. 7 - s in one MMA: the B
              // slices lie one after another in shared memory with the same
              // stride between 8-column groups, so they form one operand of
              // 32 (8 - s) columns, whose block t lands on the accumulator of
              // level s + t. The first MMA of a chunk (s = 0) covers all eight
              // levels and starts them; every other one accumulates.
#pragma unroll 1
              for (int s = 0; s < TC_SLICES; ++s)
                mma_bf16(dacc + (uint32_t)(s * TC_N), smem_desc(a0 + s * (TC_A_SLAB / TC_SLICES), 128, 256),
                         smem_desc(b0, 128, 256), mma_idesc((uint32_t)(TC_N * (TC_SLICES - s))),
                         (q == ch * SPC && s == 0) ? 0u : 1u);
              mma_commit(smem_u32(&B->empty[sg]));
            }
            mma_commit(smem_u32(&B->tfull[acc]));  // arrives once this chunk's MMAs completed
          }
      }
      // every MMA issued has completed before TMEM is released (also after an abort)
      mma_commit(smem_u32(&B->fin));
      if (!mbar_wait(smem_u32(&B->fin), 0)) p_fail(B, err, 5);
    }
  } else {
    // ---- epilogue: warp w drains TMEM lanes 32 (w mod 4) .. + 31 (rows of the
    // tile), columns EPI_COLS (w / 4) .. + EPI_COLS - 1
    const int quarter = warp & 3, cg = warp >> 2;
    const int r = quarter * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(cg * EPI_COLS);
    int u = 0;
    bool ok = true;
    for (int item = blockIdx.x; ok && item < nitems; item += gridDim.x) {
      const int slot = item / nrt, rt = item - slot * nrt;
      if (!tc_slot(st[slot].k)) continue;
      const int64_t i = (int64_t)rt * TC_M + r;
      const int e = erow[((int64_t)slot * nrt + rt) * TC_M + r];
      for (int ct = 0; ok && ct < nct; ++ct) {
        long long thi[EPI_COLS], tlo[EPI_COLS];
#pragma unroll
        for (int c = 0; c < EPI_COLS; ++c) thi[c] = tlo[c] = 0;
        for (int ch = 0; ch < nchunk; ++ch, ++u) {
          const int acc = u & 1;
          bool got = mbar_wait(smem_u32(&B->tfull[acc]), (uint32_t)((u >> 1) & 1));
          got = __all_sync(0xffffffffu, got) && !__any_sync(0xffffffffu, p_aborted(B));
          if (!got) {
            if (lane == 0) p_fail(B, err, 4);
            ok = false;
            break;
          }
          tc_fence_after();
          long long hi[EPI_COLS], lo[EPI_COLS];
#pragma unroll
          for (int c = 0; c < EPI_COLS; ++c) hi[c] = lo[c] = 0;
          // two levels per wait: the second load is in flight with the first
#pragma unroll 1
          for (int lev = 0; lev < TC_SLICES; lev += 2) {
            uint32_t v0[EPI_COLS], v1[EPI_COLS];
            tmem_ld8_async(trow + (uint32_t)(acc * 8 * TC_N + lev * TC_N), v0);
            tmem_ld8_async(trow + (uint32_t)(acc * 8 * TC_N + (lev + 1) * TC_N), v1);
            tmem_wait();
#pragma unroll
            for (int c = 0; c < EPI_COLS; ++c) {
              const long long a0 = (long long)__float2int_rn(__uint_as_float(v0[c]));
              const long long a1 = (long long)__float2int_rn(__uint_as_float(v1[c]));
              if (lev < 4) hi[c] = (hi[c] * 128 + a0) * 128 + a1;
              else lo[c] = (lo[c] * 128 + a0) * 128 + a1;
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(smem_u32(&B->tempty[acc]));  // this set may take the next chunk
#pragma unroll
          for (int c = 0; c < EPI_COLS; ++c) {
            thi[c] += hi[c];
            tlo[c] += lo[c];
          }
        }
        if (!ok || i >= n) continue;
        const int* ec = ecol + ((int64_t)slot * nct + ct) * TC_N + cg * EPI_COLS;
#pragma unroll
        for (int c = 0; c < EPI_COLS; c += 2) {
          const int j = (ct * TC_N + cg * EPI_COLS + c) >> 1;
          if (j < nf) {
            const int f0 = ec[c], f1 = ec[c + 1];
            z64 x;
            if (!int_to_double(thi[c], tlo[c], e + f0 - 35, &x.re))
              x.re = scalbn(fma((double)tlo[c], 0x1p-28, (double)thi[c]), e + f0 - 35);
            if (!int_to_double(thi[c + 1], tlo[c + 1], e + f1 - 35, &x.im))
              x.im = scalbn(fma((double)tlo[c + 1], 0x1p-28, (double)thi[c + 1]), e + f1 - 35);
            X[((int64_t)slot * nf + j) * n + i] = x;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(P_TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------ host
bool tc_supported(int K, int64_t n) { return K >= 1 && tc_slot(K) && (n + TC_M - 1) / TC_M <= 65535; }

TcLayout tc_layout(int64_t n, int nf, int K, int nslot) {
  TcLayout T{};
  T.K = K;
  T.nslab = (2 * K + TC_KSLAB - 1) / TC_KSLAB;
  T.nrt = (int)((n + TC_M - 1) / TC_M);
  T.nct = (2 * nf + TC_N - 1) / TC_N;
  T.a_bytes = (size_t)nslot * T.nrt * T.nslab * TC_A_SLAB;
  T.b_bytes = (size_t)nslot * T.nct * T.nslab * TC_B_SLAB;
  T.e_bytes = (size_t)nslot * T.nrt * TC_M * sizeof(int);
  T.f_bytes = (size_t)nslot * T.nct * TC_N * sizeof(int);
  return T;
}

size_t tc_ws_bytes(const TcLayout& T) {
  size_t need = 0;
  for (size_t b : {T.a_bytes, T.b_bytes, T.e_bytes, T.f_bytes}) need += (b + 255) & ~(size_t)255;
  return need;
}

int tc_group_size(int64_t n, int nf, int K, int nslot) {
  const size_t cap = size_t(4) << 30;
  const size_t one = tc_ws_bytes(tc_layout(n, nf, K, 1));
  const size_t g = one > 0 ? cap / one : (size_t)nslot;
  return (int)std::max<size_t>(1, std::min<size_t>((size_t)nslot, g));
}

void tc_prepare() {
  cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, P_SMEM);
}

static inline size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

int launch_tc_assemble(const TcLayout& T, const SlotState* st, const z64* Z, int64_t vsZ, const z64* Y,
                       const int32_t* mj, int nf, int m, z64* X, int64_t n, int nslot, void* ws, int* err,
                       cudaStream_t s) {
  unsigned char* w = (unsigned char*)ws;
  uint4* As = (uint4*)w;
  w += align256(T.a_bytes);
  uint4* Bs = (uint4*)w;
  w += align256(T.b_bytes);
  int* erow = (int*)w;
  w += align256(T.e_bytes);
  int* ecol = (int*)w;
  k_tc_slice_a<<<dim3(T.nrt, nslot), TC_M, 0, s>>>(st, Z, vsZ, n, T.nslab, T.nrt, As, erow);
  k_tc_slice_b<<<dim3(T.nct, nslot), TC_N, 0, s>>>(st, Y, mj, nf, m, T.nslab, T.nct, Bs, ecol);
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int items = nslot * T.nrt;
  k_tc_gemm<<<std::max(1, std::min(items, sms)), P_THREADS, P_SMEM, s>>>(
      st, (const unsigned char*)As, (const unsigned char*)Bs, erow, ecol, T.nslab, T.nrt, T.nct, n, nf, nslot, X, err);
  return 3;
}

}  // namespace fks
