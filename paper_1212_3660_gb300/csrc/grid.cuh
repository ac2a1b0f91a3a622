// Launchers of the structured-grid and multigrid kernels (grid.cu).
#pragma once
#include "common.cuh"

namespace fks {

constexpr int TAIL_THREADS = 512;
// halo of the fused level kernels: four half sweeps, one cell each
constexpr int FH = 4;

// One level of the single-block tail V-cycle; f lives at shared offset `off`
// (in complex elements) and z right after it.
template <typename T>
struct TailLevel {
  LevelView<T> L;
  int rx, ry, rz;          // ratios to the next coarser level
  const cx<T>* invd;       // [n_tau][n] inverse diagonals
  int off;
  int cbyte;               // byte offset of this level's coefficients staged in shared memory
};

template <typename T>
struct TailParams {
  int nlev;                // levels lt .. coarsest
  TailLevel<T> lev[MAX_LEVELS];
  const cx<T>* Ainv;       // [n_tau][nc][nc]
  int nc;
  uint32_t mask;
  const cx<T>* f_in;       // level-lt right-hand side (global), slot stride vs
  cx<T>* z_out;            // level-lt correction (global)
  int64_t vs;
  const z64* taus;
  int staged;              // coefficients copied to shared memory at kernel start
  const unsigned char* blob;  // staged coefficients per tau, already in the shared-memory layout (or null)
  int blob_bytes;          // bytes per tau (multiple of 16)
  int coef0;               // shared-memory byte offset of the coefficient region
  // register-resident 2D variant (tail2d_ok): every level but the coarsest is 2D,
  // halved in both axes and has at most 2 * TAIL_THREADS cells; the coarsest
  // inverse of the current tau is staged at shared byte offset ainv_off
  int pairs;
  int ainv_off;
};

template <typename T>
void tail_prepare(size_t smem_bytes);
bool fused_level_ok(const LevelHost& L);
template <typename T>
void fused_prepare();
// tile: 8, 16 or 32 (tiles of tile x tile cells); the results do not depend on the tiling
template <typename T>
void launch_pre2d(const LevelHost& F, const LevelHost& C, const SlotState* st, const cx<T>* invd, const z64* taus,
                  const cx<T>* f, cx<T>* z, int64_t vs, cx<T>* fc, int64_t vsc, int nslot, int tile, cudaStream_t s);
// Zk (optional): instead of writing zout, add the result to column k - 1 of the
// outer iterates Zk (slot stride vsZk, column stride zcol), as launch_correct does.
template <typename T>
void launch_post2d(const LevelHost& F, const LevelHost& C, uint32_t mask, const SlotState* st, const cx<T>* invd,
                   const cx<T>* f, const cx<T>* z, cx<T>* zout, int64_t vs, const cx<T>* zc, int64_t vsc, int nslot,
                   int tile, cudaStream_t s, z64* Zk = nullptr, int64_t vsZk = 0, int64_t zcol = 0);
// 3D levels coarsened by 2 in every axis (grid3d.cu): tile 8 (8 x 8), 16
// (16 x 16) or 32 (32 x 16) cells in x-y, zc planes per block (even; <= 0: all)
bool fused3d_level_ok(const LevelHost& L);
template <typename T>
void fused3d_prepare();
template <typename T>
void launch_pre3d(const LevelHost& F, const SlotState* st, const cx<T>* invd, const z64* taus, const cx<T>* f,
                  cx<T>* z, int64_t vs, cx<T>* fc, int64_t vsc, int nslot, int tile, int zc, cudaStream_t s);
template <typename T>
void launch_post3d(const LevelHost& F, uint32_t mask, const SlotState* st, const cx<T>* invd, const cx<T>* f,
                   const cx<T>* z, cx<T>* zout, int64_t vs, const cx<T>* zc, int64_t vsc, int nslot, int tile,
                   int zch, cudaStream_t s, z64* Zk = nullptr, int64_t vsZk = 0, int64_t zcol = 0);
// P.pairs selects the register-resident 2D kernel (same results)
template <typename T>
void launch_tail(const TailParams<T>& P, size_t smem_bytes, const SlotState* st, int nslot, cudaStream_t s);
// whether levels lt .. coarsest qualify for the register-resident 2D tail
bool tail2d_ok(const std::vector<LevelHost>& Ls, int lt);

void launch_faces_from_cond(const LevelHost& L, const double h[3], uint32_t mask, const double* cond, cudaStream_t s);
void launch_coarsen(const LevelHost& F, const LevelHost& C, const double* fac_x, const double* fac_y,
                    const double* fac_z, cudaStream_t s);
// Factors of the coarse faces along one axis (index 0..nc: the face below
// coarse cell I; nc: the high boundary): fine centre distance across the face
// over the coarse one, from the fine cells' widths w in finest cells (half
// widths at the boundary); 1/2 everywhere on evenly halved axes, 1 where r = 1.
// W receives the coarse widths.
std::vector<double> coarse_face_factors(const std::vector<double>& w, int r, std::vector<double>* W);
void launch_to_f32(const double* a, float* b, int64_t n, cudaStream_t s);
// from_f32: from the level's fp32 coefficients (the bf16-smoother option's
// rounded values) instead of its fp64 ones
template <typename T>
void launch_invd(const LevelHost& L, const z64* taus, int ntau, cx<T>* out, cudaStream_t s, int from_f32 = 0);
void launch_coarse_inverse(const LevelHost& L, const z64* taus, int ntau, z64* work, z64* inv, int* singular,
                           cudaStream_t s, int from_f32 = 0);
// b = a rounded to bf16, r = the same value as fp32
void launch_round_bf16(const double* a, __nv_bfloat16* b, float* r, int64_t n, cudaStream_t s);
template <typename T>
void launch_to_prec(const z64* a, cx<T>* b, int64_t n, cudaStream_t s);
template <typename T>
void launch_apply(const LevelHost& L, z64 sfix, const SlotState* st, const z64* taus, const cx<T>* x, cx<T>* y,
                  int64_t vs, int nslot, cudaStream_t s);
// Zk (optional): the finest level's last half sweep, fused with the defect
// correction (both cells of each pair are added to column k - 1 of Zk, as
// launch_correct does; z is not written)
template <typename T>
void launch_gs(const LevelHost& L, const SlotState* st, const cx<T>* invd, const cx<T>* f, cx<T>* z, int64_t vs,
               int nslot, int color, int zero_start, cudaStream_t s, z64* Zk = nullptr, int64_t vsZk = 0,
               int64_t zcol = 0, int bf16 = 0);
template <typename T>
void launch_residual_restrict(const LevelHost& F, const LevelHost& C, const SlotState* st, const z64* taus,
                              const cx<T>* f, const cx<T>* z, int64_t vs, cx<T>* fc, int64_t vsc, int nslot,
                              cudaStream_t s, int bf16 = 0);
template <typename T>
void launch_prolong_add(const LevelHost& F, const LevelHost& C, uint32_t mask, const SlotState* st, const cx<T>* zc,
                        int64_t vsc, cx<T>* z, int64_t vs, int nslot, cudaStream_t s);
template <typename T>
void launch_coarse_solve(const cx<T>* Ainv, int n, const SlotState* st, const cx<T>* f, cx<T>* z, int64_t vs,
                         int nslot, cudaStream_t s);
template <typename T>
void launch_correct(const SlotState* st, z64* z, int64_t zs, int64_t zcol, const cx<T>* e, int64_t es, int64_t n,
                    int nslot, cudaStream_t s);
int defect_blocks(const LevelHost& L);
template <typename T>
void launch_defect(const LevelHost& L, const SlotState* st, const z64* taus, const z64* v, int64_t vsv, const z64* z,
                   int64_t vsz, int64_t col, int zero_z, cx<T>* f0, int64_t vsf, double* partial, int with_v,
                   int nslot, cudaStream_t s);
// The defect of launch_defect with the inner-solve decision of
// launch_inner_decide taken by the last block of each slot (one launch);
// bcount: nslot zero ints, left zero.
// diag64: [n_tau][n] K_cc + tau M_cc of this level (launch_diag64), or null.
template <typename T>
void launch_defect_decide(const LevelHost& L, SlotState* st, const z64* taus, const z64* diag64, const z64* v,
                          int64_t vsv, const z64* z, int64_t vsz, int64_t col, int zero_z, cx<T>* f0, int64_t vsf,
                          double* partial, double eps, int max_cycles, const int32_t* replay_cycles, int m_max,
                          int use_cond, cudaGraphConditionalHandle cond, int* flags, int* counter, int* bcount,
                          int nslot, double relax, double tol, cudaStream_t s);
void launch_diag64(const LevelHost& L, const z64* taus, int ntau, z64* out, cudaStream_t s);
// kd[c] = sum of the faces of cell c (the diagonal of K) in fp64
void launch_kdiag(const LevelHost& L, double* kd, cudaStream_t s);
void launch_inner_decide(SlotState* st, int nslot, const double* partial, int nblocks, int first, double eps,
                         int max_cycles, const int32_t* replay_cycles, int m_max, int use_cond,
                         cudaGraphConditionalHandle cond, int* flags, int* counter, cudaStream_t s,
                         double relax = 0.0, double tol = 0.0);

}  // namespace fks
