// The lower part of a multigrid V-cycle in one thread-block cluster per source
// (cluster.cu): every 2D level from a starting level down to the level above
// the coarsest is split into CL_SIZE bands of rows, band b living in the shared
// memory of CTA b with its coefficients; rows across a band edge are read from
// the neighbouring CTA's shared memory (distributed shared memory) and the
// half sweeps are separated by cluster barriers. The coarsest level is solved
// by its dense inverse in CTA 0. Every cell update performs the operations of
// the per-level kernels in the same order, so results do not depend on whether
// this kernel runs.
#pragma once
#include "common.cuh"

namespace fks {

constexpr int CL_SIZE = 8;         // CTAs per cluster (portable cluster size)
constexpr int CL_THREADS = 512;
constexpr int CL_MAX_LEVELS = 10;
constexpr int CL_MAX_COARSE = 64;  // coarsest level solved by one CTA
constexpr size_t CL_SMEM_LIMIT = 200 * 1024;

// One banded level; byte offsets into the shared memory of every CTA.
struct ClLevel {
  int nx, ny, R;             // R = ny / CL_SIZE rows per band
  int f, z;                  // right-hand side and iterate (R x nx complex)
  int fx, fy, mm, id;        // coefficients of the band: R x (nx+1), (R+1) x nx, R x nx, R x nx complex
};

template <typename T>
struct ClusterParams {
  int nlev;                  // banded levels
  ClLevel lev[CL_MAX_LEVELS];
  int ncx, ncy, nc;          // coarsest level
  int fC, zC;                // its f and z (used in CTA 0)
  int rs;                    // residuals of the last banded level (restricted by CTA 0)
  int ainv;                  // its dense inverse, staged with the coefficients
  uint32_t mask;             // zero-head faces
  const cx<T>* f_in;         // right-hand side of the first banded level (global), slot stride vs
  cx<T>* z_out;              // its correction (global)
  int64_t vs;
  const unsigned char* blob; // per tau: CL_SIZE regions of `region` bytes (band coefficients + inverse)
  int region;
  int coef0;                 // shared-memory offset the region is copied to
  const z64* taus;
};

// Host-side layout of the cluster part for levels [l0, L): false if it does not
// apply (3D level, a level not halved in both axes, rows not a multiple of
// CL_SIZE, coarsest level too large, shared memory exceeded).
template <typename T>
bool cluster_layout(const std::vector<LevelHost>& Ls, int l0, ClusterParams<T>* P, size_t* smem_bytes);
// The per-tau coefficient regions of every CTA (levels of P, the coarsest
// inverse Ainv [n_tau][nc][nc]); blob holds n_tau * CL_SIZE * P.region bytes.
template <typename T>
void launch_cluster_blob(const std::vector<LevelHost>& Ls, int l0, const ClusterParams<T>& P, const cx<T>* const* invd,
                         const cx<T>* Ainv, int ntau, unsigned char* blob, cudaStream_t s);
template <typename T>
void cluster_prepare(size_t smem_bytes);
template <typename T>
void launch_cluster_vcycle(const ClusterParams<T>& P, size_t smem_bytes, const SlotState* st, int nslot,
                           cudaStream_t s);
// whether clusters of this kernel with this shared memory can be scheduled
template <typename T>
bool cluster_launchable(size_t smem_bytes);

}  // namespace fks
