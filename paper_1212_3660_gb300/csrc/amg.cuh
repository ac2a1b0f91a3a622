// Smoothed-aggregation algebraic multigrid for K + tau M (amg.cu): the host
// setup of one tau's hierarchy and the V-cycle that preconditions the BiCGSTAB
// steps of a CSR operator's inner solve (Section 6).
#pragma once
#include <string>
#include <vector>

#include "common.cuh"

namespace fks {

constexpr int AMG_MAX_LEVELS = 16;
constexpr int64_t AMG_MAX_DENSE = 4096;  // largest coarsest level (dense inverse)

// One level of one tau's hierarchy on the device, values in the cycle precision T.
template <typename T>
struct AmgLevel {
  int64_t n, nc;                  // unknowns of this level and of the next (0 on the coarsest)
  const int64_t* arp;             // A_l (level 0: K + tau M on the entries where K or M is nonzero)
  const int32_t* aci;
  const cx<T>* av;
  const cx<T>* dinv;              // 1 / diag(A_l)
  T omega;                        // Jacobi weight 4 / (3 rho_l)
  const int64_t* prp;             // P_l, n x nc
  const int32_t* pci;
  const cx<T>* pv;
  const int64_t* rrp;             // R_l = P_l^T, nc x n
  const int32_t* rci;
  const cx<T>* rv;
  const cx<T>* cinv;              // coarsest level: dense inverse, row-major n x n
};

// ---------------------------------------------------------------- host setup
struct AmgCsr {                   // complex128 CSR, columns sorted within a row
  int64_t n = 0, m = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<z64> v;
};

struct AmgHostLevel {
  AmgCsr A, P, R;
  std::vector<z64> dinv;
  double omega = 0.0;
};

struct AmgHost {
  std::vector<AmgHostLevel> lv;
  std::vector<z64> cinv;          // dense inverse of the coarsest A (row-major)
};

// Aggregates of every level but the coarsest. They depend on the sparsity
// pattern only, so the first tau's build fixes them for every other tau.
struct AmgAgg {
  std::vector<std::vector<int32_t>> agg;
  std::vector<int32_t> count;
};

// The hierarchy of A0 (level 0; its pattern is the strength graph). With
// agg->agg empty the aggregates are computed and stored; otherwise they are
// reused and fix the number of levels. Returns "" or an error message.
std::string amg_build(const AmgCsr& A0, int max_levels, int64_t max_coarse, AmgAgg* agg, AmgHost* out);

// Device copies of a host hierarchy in precision T: every allocation is
// appended to `mem` (the caller frees them, also after an error), one
// AmgLevel per level to `levels`.
template <typename T>
cudaError_t amg_upload(const AmgHost& h, std::vector<void*>& mem, std::vector<AmgLevel<T>>& levels);

// ---------------------------------------------------------------- V-cycle
// Per-level work vectors of a batch ([nslot][n_l] each, cycle precision) and
// the device table of the batch's hierarchies: tab[tau * L + l].
template <typename T>
struct AmgRun {
  const AmgLevel<T>* tab;
  int L, nu;
  int64_t n[AMG_MAX_LEVELS];
  cx<T>* f[AMG_MAX_LEVELS];       // right-hand side of level l >= 1
  cx<T>* x[AMG_MAX_LEVELS];       // iterate
  cx<T>* y[AMG_MAX_LEVELS];       // second Jacobi buffer
  cx<T>* r[AMG_MAX_LEVELS];       // residual, then (l >= 1) the level's result
};

struct BcgScal;
struct SlotState;

#ifdef __CUDACC__
// Per-row arithmetic of the V-cycle, shared by the stage kernels (amg.cu) and
// the cooperative cycle (csr.cu) so that both give the same bits. Vectors are
// read through L2 (__ldcg): in the cooperative kernel other blocks wrote them
// before the last grid barrier.
template <typename T>
__device__ __forceinline__ cx<T> amg_ld(const cx<T>* p) {
  if constexpr (sizeof(T) == 8) {
    const double2 v = __ldcg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
  } else {
    const float2 v = __ldcg(reinterpret_cast<const float2*>(p));
    return mk(v.x, v.y);
  }
}

// sum_q v_q x[col_q] over one CSR row
template <typename T>
__device__ __forceinline__ cx<T> amg_row(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                         const cx<T>* __restrict__ v, int64_t row, const cx<T>* x) {
  cx<T> acc = mk(T(0), T(0));
  for (int64_t q = rp[row]; q < rp[row + 1]; ++q) acc = acc + v[q] * amg_ld(x + ci[q]);
  return acc;
}

// first sweep from zero: omega D^{-1} f at row i (elementwise; its producer computes it)
template <typename T>
__device__ __forceinline__ cx<T> amg_first(const AmgLevel<T>& A, int64_t i, cx<T> f) {
  return A.omega * (A.dinv[i] * f);
}

// a later sweep: x_i + omega D^{-1} (f - A x)_i
template <typename T>
__device__ __forceinline__ cx<T> amg_sweep(const AmgLevel<T>& A, int64_t i, const cx<T>* f, const cx<T>* x) {
  const cx<T> ax = amg_row(A.arp, A.aci, A.av, i, x);
  return amg_ld(x + i) + A.omega * (A.dinv[i] * (amg_ld(f + i) - ax));
}

// (f - A x)_i
template <typename T>
__device__ __forceinline__ cx<T> amg_resid(const AmgLevel<T>& A, int64_t i, const cx<T>* f, const cx<T>* x) {
  return amg_ld(f + i) - amg_row(A.arp, A.aci, A.av, i, x);
}

// row `row` of the coarsest level's dense inverse times f, by one warp (lanes
// over columns, fixed-order shuffle reduction); the sum is valid in lane 0
template <typename T>
__device__ __forceinline__ cx<T> amg_coarse_row(const AmgLevel<T>& A, int64_t row, const cx<T>* f, int lane) {
  const int64_t n = A.n;
  cx<T> acc = mk(T(0), T(0));
  for (int64_t j = lane; j < n; j += 32) acc = acc + A.cinv[row * n + j] * amg_ld(f + j);
  for (int s = 16; s > 0; s >>= 1) {
    acc.re += __shfl_down_sync(0xffffffffu, acc.re, s);
    acc.im += __shfl_down_sync(0xffffffffu, acc.im, s);
  }
  return acc;
}
#endif

// out0 = V_0(f0) for every slot whose inner solve runs and whose BiCGSTAB
// cycle has not halted (sc may be null); returns the number of launches. The
// first sweep of level 0, R.x[0] = omega_0 D_0^{-1} f0, must already be there:
// the kernel that produces f0 writes it.
template <typename T>
int launch_amg_vcycle(const AmgRun<T>& R, const SlotState* st, const BcgScal* sc, const cx<T>* f0, cx<T>* out0,
                      int nslot, cudaStream_t s);

}  // namespace fks
