// Launchers of the Krylov kernels (krylov.cu).
#pragma once
#include "common.cuh"

namespace fks {

constexpr int MD_THREADS = 256;  // threads per block of the multi-dot kernel
constexpr int MD_ROWS = 16;      // rows per thread
constexpr int MD_COLS = 16;      // basis columns per block
constexpr int GV_WARPS = 4;      // shifts per block of the Givens kernel
constexpr int AS_J = 8;          // shifts per block of the assembly kernel
constexpr int TRES_ROWS = 2;     // rows of cells per thread in the true-residual kernel

int norm_blocks(int64_t n);
int mdot_blocks(int64_t n);
int tres_blocks(const LevelHost& L);

void launch_norm2_partial(const SlotState* st, int need_active, const z64* x, int64_t vs, int64_t n, double* partial,
                          int nslot, cudaStream_t s);
void launch_start(SlotState* st, int nslot, const double* partial, int nblocks, int nf, cudaStream_t s);
// V32 (optional): also the complex64 copy of v_1
void launch_init_v1(const SlotState* st, const z64* b, int64_t n, z64* V, int64_t vsV, int nslot, cudaStream_t s,
                    z32* V32 = nullptr);
void launch_init_shifts(const SlotState* st, int nf, int m, int32_t* sst, int32_t* mj, double* est, double* bnd,
                        z64* Y, double* alpha, int nslot, cudaStream_t s);
void launch_step_begin(SlotState* st, int nslot, const int32_t* sched, int sched_len, const z64* taus, z64* taus_k,
                       int m, cudaStream_t s);
void launch_mass(const SlotState* st, const double* mm, const z64* Z, int64_t vsZ, z64* w, int64_t n, double* partial,
                 int nslot, cudaStream_t s);
void launch_mdot(const SlotState* st, const z64* V, int64_t vsV, const z64* w, int64_t n, z64* partial, int kmax,
                 int nslot, cudaStream_t s);
// the first CGS projection from the complex64 copy of the basis (fp32 sums)
void launch_mdot32(const SlotState* st, const z32* V, int64_t vsV, const z64* w, int64_t n, z64* partial, int kmax,
                   int nslot, cudaStream_t s);
void launch_hreduce(const SlotState* st, const z64* partial, int64_t n, z64* h, int64_t hstride, int nslot,
                    cudaStream_t s);
void launch_maxpy(const SlotState* st, const z64* V, int64_t vsV, const z64* h, int64_t hstride, z64* w, int64_t n,
                  int nslot, cudaStream_t s);
void launch_arnoldi_finish(SlotState* st, int nslot, const z64* h12, const double* wpart, const double* mpart,
                           int nblocks, z64* H, int m, double* pn, int32_t* cyc, double rtol, cudaStream_t s);
void launch_new_v(const SlotState* st, const z64* w, int64_t n, const z64* H, int m, z64* V, int64_t vsV, int nslot,
                  cudaStream_t s, z32* V32 = nullptr);
void launch_givens(SlotState* st, int nf, int m, const z64* sigma, const z64* H, const z64* taus_k, const double* pn,
                   double tol, int variant, const int32_t* replay_mj, z64* g, double* rc, z64* rs, z64* R, z64* Y,
                   int32_t* sst, int32_t* mj, double* est, double* bnd, double* alpha, int nslot, cudaStream_t s,
                   const double* tol_shift = nullptr, z64* coef = nullptr);
// budget (optional, device): steps left in this launch of the step loop
void launch_step_end(SlotState* st, int nslot, int m, int use_cond, cudaGraphConditionalHandle cond, cudaStream_t s,
                     int* budget = nullptr);
// st[slot].active = 0 where stop[slot] != 0
void launch_stop_slots(SlotState* st, const int* stop, int nslot, cudaStream_t s);
// x_j = Z y_j in FP64; with st given, sources with st[slot].k <= skip_k_le are skipped
void launch_assemble(const z64* Z, int64_t vsZ, const z64* Y, const int32_t* mj, int nf, int m, z64* X, int64_t n,
                     int nslot, cudaStream_t s, const SlotState* st = nullptr, int skip_k_le = -1);
void launch_true_residual(const LevelHost& L, const z64* sigma, int nf, const z64* b, const z64* X, double* partial,
                          const SlotState* st, double* out, int nslot, cudaStream_t s);

// out[slot * nf + j] = sqrt(sum of the nblocks partials) / beta_slot
// X[idx[i]] += a[i] Xh[idx[i]] (columns of n), i < ncols
void launch_axpy_cols(z64* X, const z64* Xh, const int32_t* idx, const z64* a, int ncols, int64_t n, cudaStream_t s);
void launch_tres_finish(const SlotState* st, const double* partial, int nblocks, int nf, int nslot, double* out,
                        cudaStream_t s);

}  // namespace fks
