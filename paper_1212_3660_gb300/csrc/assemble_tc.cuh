// Assembly X = Z Y (Algorithm 4, x_j = Z_{m_j} y_j) on the tcgen05 tensor cores.
//
// Z (n x K complex128 per source) and Y (K x n_f) are turned into one real
// product C = A B with A = [Re z_k, Im z_k]_k (n x 2K) and, for shift j, the
// columns 2j = [Re y; -Im y] and 2j+1 = [Im y; Re y] interleaved over k, so that
// C[:, 2j] = Re x_j and C[:, 2j+1] = Im x_j. Every row of A and every column of
// B is scaled by a power of two below 1 in magnitude and cut into eight signed
// 7-bit integer slices (56 bits), which bf16 holds exactly. The products of
// slices s and t with s + t <= 9 are accumulated on the tensor cores in fp32,
// one TMEM accumulator per level s + t, over chunks of at most 128 k' (64
// Arnoldi steps): every partial sum is an integer below 2^24 (at most 8 pairs x
// 127^2 x 128 terms), so the accumulation is exact. After each chunk the
// epilogue adds the levels into 64-bit integer totals; after the last it scales
// once in double. Sources of up to 128 steps (two chunks) are assembled here.
// The dropped levels and the truncated digits leave an error below
// 2^-49 max|A_i.| max|B_.j| per entry, at the level of an FP64 GEMM.
#pragma once
#include "common.cuh"

namespace fks {

constexpr int TC_SLICES = 8;      // 7-bit slices per value
constexpr int TC_M = 128;         // rows of a tile (TMEM lanes)
constexpr int TC_N = 32;          // real columns of a tile (16 shifts)
constexpr int TC_KSLAB = 16;      // k' per MMA (bf16)
constexpr int TC_CHUNK_KP = 128;  // exactness bound of one TMEM accumulation (padded k')
constexpr int TC_MAX_KP = 256;    // padded 2K of the largest source (two chunks; MAX_M = 128 steps)
constexpr int TC_A_SLAB = TC_SLICES * TC_M * TC_KSLAB * 2;  // bytes of one slab of A slices (32 KB)
constexpr int TC_B_SLAB = TC_SLICES * TC_N * TC_KSLAB * 2;  // bytes of one slab of B slices (8 KB)

struct TcLayout {
  int K;        // Arnoldi steps (complex columns of Z used)
  int nslab;    // padded 2K / 16
  int nrt;      // row tiles
  int nct;      // column tiles (2 n_f / 32, rounded up)
  size_t a_bytes, b_bytes, e_bytes, f_bytes;
};

TcLayout tc_layout(int64_t n, int nf, int K, int nslot);
// Bytes of the workspace a layout needs (a, b, e, f, each 256-byte aligned).
size_t tc_ws_bytes(const TcLayout& T);
// Sources assembled per launch group: all of them while their slices take at
// most 4 GiB, else as many as fit (at least one), so that the slice workspace
// stays bounded for large batches.
int tc_group_size(int64_t n, int nf, int K, int nslot);
// 2K padded to 16 within the exactness bound, and the row tiles within a grid dimension
bool tc_supported(int K, int64_t n);
void tc_prepare();
// Slices and exponents, then the tensor-core product and the epilogue, for the
// sources whose own step count st[slot].k is at most TC_MAX_KP / 2 = 128 (the others
// are left to the FP64 kernel); T.K is the largest such count. `ws` holds the
// layout's bytes (a, b, e, f). Returns the number of kernels launched.
int launch_tc_assemble(const TcLayout& T, const SlotState* st, const z64* Z, int64_t vsZ, const z64* Y,
                       const int32_t* mj, int nf, int m, z64* X, int64_t n, int nslot, void* ws, int* err,
                       cudaStream_t s);

}  // namespace fks
