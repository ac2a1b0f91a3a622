// Launchers of the general sparse (CSR) kernels (csr.cu).
#pragma once
#include "common.cuh"

namespace fks {
template <typename T>
struct AmgRun;
}

namespace fks {

// K + s M on the union pattern of K and M: one column index and a K and an M
// value per stored entry (zero where a matrix has no entry), in sliced ELL
// order: the rows are cut into slices of CSR_SLICE consecutive rows, and
// entry q of row r sits at sell[r / CSR_SLICE] + q * CSR_SLICE + r % CSR_SLICE
// (q < len[r], a row's entries in ascending column order). Threads that own
// consecutive rows then read consecutive addresses for each q.
constexpr int CSR_SLICE = 32;

template <typename T>
struct CsrView {
  int64_t n;
  const int64_t* sell;  // [n / CSR_SLICE + 1] start of each slice
  const int32_t* len;   // [n] entries of each row
  const int32_t* col;
  const T* kv;
  const T* mv;
};

// position of entry q of row `row`
template <typename T>
__device__ __forceinline__ int64_t csr_at(const CsrView<T>& A, int64_t row, int q) {
  return A.sell[row / CSR_SLICE] + (int64_t)q * CSR_SLICE + (row % CSR_SLICE);
}

// BiCGSTAB work vectors of the sources, each [nslot][n] in the cycle precision.
template <typename T>
struct BcgVecs {
  cx<T>* f;   // right-hand side of the cycle (the defect)
  cx<T>* e;   // result of the cycle
  cx<T>* r;
  cx<T>* rh;
  cx<T>* p;
  cx<T>* v;
  cx<T>* ph;
  cx<T>* s;
  cx<T>* sh;
  cx<T>* t;
};

struct BcgScal {
  z64 rho_old, rho, alpha, omega, beta;
  int halt, last;
};

// blocks of the grid-stride CSR kernels that write per-block partial sums
int csr_blocks(int64_t n);
template <typename T>
void launch_csr_apply(const CsrView<T>& A, z64 sfix, const SlotState* st, const z64* taus, const cx<T>* x, cx<T>* y,
                      int64_t vs, int nslot, cudaStream_t s);
template <typename T>
void launch_csr_defect(const CsrView<double>& A, const SlotState* st, const z64* taus, const z64* v, int64_t vsv,
                       const z64* z, int64_t vsz, int64_t col, int zero_z, cx<T>* f0, int64_t vsf, double* partial,
                       int nslot, cudaStream_t s);
void launch_csr_mass(const CsrView<double>& A, const SlotState* st, const z64* Z, int64_t vsZ, z64* w, double* partial,
                     int nslot, cudaStream_t s);
// ||b - (K + sigma_j M) x_j|| / ||b|| per source and shift; partial holds
// nslot * nf * csr_blocks(n) doubles
void launch_csr_true_residual(const CsrView<double>& A, const z64* sigma, int nf, const z64* b, const z64* X,
                              double* partial, const SlotState* st, double* out, int nslot, cudaStream_t s);
template <typename T>
void launch_csr_dinv(int64_t n, const double* dk, const double* dm, const z64* taus, int ntau, cx<T>* out,
                     cudaStream_t s);
template <typename T>
void launch_bcg_cycle(const CsrView<T>& A, const SlotState* st, const z64* taus, const BcgVecs<T>& V,
                      const cx<T>* dinv, BcgScal* sc, double* partial, int steps, int nslot, cudaStream_t s,
                      int* launches);
// the same cycle preconditioned by the AMG V-cycle of R (amg.cuh); with
// g_bcg_amg_coop = 0 always as stage kernels (the cooperative launch computes
// the same bits)
extern int g_bcg_amg_coop;
template <typename T>
void launch_bcg_cycle_amg(const CsrView<T>& A, const SlotState* st, const z64* taus, const BcgVecs<T>& V,
                          const AmgRun<T>& R, BcgScal* sc, double* partial, int steps, int nslot, cudaStream_t s,
                          int* launches);

}  // namespace fks
