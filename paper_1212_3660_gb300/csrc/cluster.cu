// Lower part of the V-cycle in one thread-block cluster per source (see
// cluster.cuh). The operations on every cell are those of k_gs / k_pre2d /
// k_post2d / k_tail_vcycle in the same order:
//   Gauss-Seidel   z = invd * (f + t_xl z_xl + t_xh z_xh + t_yl z_yl + t_yh z_yh)
//   residual       f - ((d + tau m) z - sum t z_nb), d the sum of the cell's faces
//   restriction    sum of the four children's residuals, children in (y, x) order
//   prolongation   prolong_value_at (cell-centred bilinear)
//   coarsest       z = Ainv f, row by row.
#include <cooperative_groups.h>

#include "cluster.cuh"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace fks {

namespace {

__device__ __forceinline__ bool cl_running(const SlotState* st, int slot) {
  return st == nullptr || (st[slot].active && !st[slot].inner_done);
}

inline size_t al16(size_t b) { return (b + 15) & ~(size_t)15; }

}  // namespace

template <typename T>
bool cluster_layout(const std::vector<LevelHost>& Ls, int l0, ClusterParams<T>* P, size_t* smem_bytes) {
  const int L = (int)Ls.size();
  if (l0 < 0 || l0 >= L - 1) return false;
  const int nlev = L - 1 - l0;
  if (nlev > CL_MAX_LEVELS) return false;
  ClusterParams<T> Q{};
  Q.nlev = nlev;
  for (int l = l0; l < L - 1; ++l) {
    const LevelHost& A = Ls[l];
    if (A.nz != 1 || A.rx != 2 || A.ry != 2 || A.rz != 1 || A.nx % 2 || A.ny % 2) return false;
    if (A.ny % CL_SIZE != 0) return false;
    const int R = A.ny / CL_SIZE;
    // a banded coarser level must take exactly the two fine rows of each coarse row
    if (l + 1 < L - 1 && (R % 2 != 0)) return false;
    Q.lev[l - l0].nx = A.nx;
    Q.lev[l - l0].ny = A.ny;
    Q.lev[l - l0].R = R;
  }
  const LevelHost& C = Ls[L - 1];
  if (C.nz != 1 || C.n > CL_MAX_COARSE) return false;
  Q.ncx = C.nx;
  Q.ncy = C.ny;
  Q.nc = (int)C.n;
  const size_t c = sizeof(cx<T>), r = sizeof(T);
  size_t off = 0;
  for (int i = 0; i < nlev; ++i) {
    ClLevel& A = Q.lev[i];
    const size_t cells = (size_t)A.R * A.nx;
    A.f = (int)off;
    off = al16(off + cells * c);
    A.z = (int)off;
    off = al16(off + cells * c);
  }
  Q.fC = (int)off;
  off = al16(off + (size_t)Q.nc * c);
  Q.zC = (int)off;
  off = al16(off + (size_t)Q.nc * c);
  // residuals of the last banded level (its restriction crosses bands)
  const ClLevel last = Q.lev[nlev - 1];
  Q.rs = (int)off;
  off = al16(off + (size_t)last.R * last.nx * c);
  Q.coef0 = (int)off;
  for (int i = 0; i < nlev; ++i) {
    ClLevel& A = Q.lev[i];
    A.fx = (int)off;
    off = al16(off + (size_t)A.R * (A.nx + 1) * r);
    A.fy = (int)off;
    off = al16(off + (size_t)(A.R + 1) * A.nx * r);
    A.mm = (int)off;
    off = al16(off + (size_t)A.R * A.nx * r);
    A.id = (int)off;
    off = al16(off + (size_t)A.R * A.nx * c);
  }
  Q.ainv = (int)off;
  off = al16(off + (size_t)Q.nc * Q.nc * c);
  Q.region = (int)(off - Q.coef0);
  if (off > CL_SMEM_LIMIT) return false;
  *P = Q;
  *smem_bytes = off;
  return true;
}

template <typename T>
struct ClBlobArgs {
  int nlev;
  const T* fx[CL_MAX_LEVELS];
  const T* fy[CL_MAX_LEVELS];
  const T* mm[CL_MAX_LEVELS];
  const cx<T>* id[CL_MAX_LEVELS];
  int64_t n[CL_MAX_LEVELS];
  const cx<T>* ainv;
};

template <typename T>
__global__ void k_cluster_blob(ClusterParams<T> P, ClBlobArgs<T> A, unsigned char* blob) {
  const int b = blockIdx.x, q = blockIdx.y;
  unsigned char* dst = blob + ((size_t)q * CL_SIZE + b) * P.region;  // shared offset o -> dst + (o - coef0)
  for (int l = 0; l < P.nlev; ++l) {
    const ClLevel L = P.lev[l];
    T* fx = (T*)(dst + (L.fx - P.coef0));
    T* fy = (T*)(dst + (L.fy - P.coef0));
    T* mm = (T*)(dst + (L.mm - P.coef0));
    cx<T>* id = (cx<T>*)(dst + (L.id - P.coef0));
    const int64_t r0 = (int64_t)b * L.R;
    for (int t = threadIdx.x; t < L.R * (L.nx + 1); t += blockDim.x) fx[t] = A.fx[l][r0 * (L.nx + 1) + t];
    for (int t = threadIdx.x; t < (L.R + 1) * L.nx; t += blockDim.x) fy[t] = A.fy[l][r0 * L.nx + t];
    for (int t = threadIdx.x; t < L.R * L.nx; t += blockDim.x) {
      mm[t] = A.mm[l][r0 * L.nx + t];
      id[t] = A.id[l][(int64_t)q * A.n[l] + r0 * L.nx + t];
    }
  }
  cx<T>* ai = (cx<T>*)(dst + (P.ainv - P.coef0));
  for (int t = threadIdx.x; t < P.nc * P.nc; t += blockDim.x) ai[t] = A.ainv[(int64_t)q * P.nc * P.nc + t];
}

template <typename T>
__global__ void __cluster_dims__(CL_SIZE, 1, 1) __launch_bounds__(CL_THREADS, 1)
    k_cluster_vcycle(ClusterParams<T> P, const SlotState* st) {
  cg::cluster_group cl = cg::this_cluster();
  const int b = (int)cl.block_rank();
  const int slot = blockIdx.x / CL_SIZE;
  if (!cl_running(st, slot)) return;  // the same for every CTA of the cluster
  extern __shared__ __align__(16) unsigned char csm[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int tau = st[slot].tau;
  const cx<T> sft = cvt<T>(P.taus[tau]);
  {
    const uint4* src = (const uint4*)(P.blob + ((size_t)tau * CL_SIZE + b) * P.region);
    uint4* dst = (uint4*)(csm + P.coef0);
    for (int q = tid; q < P.region / 16; q += nt) dst[q] = src[q];
    const ClLevel A = P.lev[0];
    cx<T>* F = (cx<T>*)(csm + A.f);
    const cx<T>* fin = P.f_in + slot * P.vs + (int64_t)b * A.R * A.nx;
    for (int q = tid; q < A.R * A.nx; q += nt) F[q] = fin[q];
  }
  cl.sync();

  // z of the row just above (below) this band at level A: the last (first) row
  // of the neighbouring CTA's band
  auto zrow = [&](const ClLevel A, cx<T>* Z, int lj, int i) -> cx<T> {
    if (lj < 0) return cl.map_shared_rank(Z, b - 1)[(A.R - 1) * A.nx + i];
    if (lj >= A.R) return cl.map_shared_rank(Z, b + 1)[i];
    return Z[lj * A.nx + i];
  };
  auto sweep = [&](const ClLevel A, int color, int zs) {
    const cx<T>* F = (const cx<T>*)(csm + A.f);
    cx<T>* Z = (cx<T>*)(csm + A.z);
    const T* FX = (const T*)(csm + A.fx);
    const T* FY = (const T*)(csm + A.fy);
    const cx<T>* ID = (const cx<T>*)(csm + A.id);
    const int nxh = (A.nx + 1) >> 1;
    for (int t = tid; t < A.R * nxh; t += nt) {
      const int lj = t / nxh, ii = t - lj * nxh;
      const int j = b * A.R + lj;
      const int i = 2 * ii + ((j + color) & 1);
      if (i >= A.nx) continue;
      const int r = lj * A.nx + i;
      cx<T> rhs = F[r];
      if (!zs) {
        const T xl = FX[lj * (A.nx + 1) + i], xh = FX[lj * (A.nx + 1) + i + 1];
        const T yl = FY[lj * A.nx + i], yh = FY[(lj + 1) * A.nx + i];
        if (i > 0) rhs = axpy(xl, Z[r - 1], rhs);
        if (i < A.nx - 1) rhs = axpy(xh, Z[r + 1], rhs);
        if (j > 0) rhs = axpy(yl, zrow(A, Z, lj - 1, i), rhs);
        if (j < A.ny - 1) rhs = axpy(yh, zrow(A, Z, lj + 1, i), rhs);
      }
      Z[r] = ID[r] * rhs;
    }
    cl.sync();
  };
  // f - (K + tau M) z at local cell (i, lj) of level A
  auto residual = [&](const ClLevel A, int i, int lj) -> cx<T> {
    const cx<T>* F = (const cx<T>*)(csm + A.f);
    cx<T>* Z = (cx<T>*)(csm + A.z);
    const T* FX = (const T*)(csm + A.fx);
    const T* FY = (const T*)(csm + A.fy);
    const T* MM = (const T*)(csm + A.mm);
    const int j = b * A.R + lj, r = lj * A.nx + i;
    Faces<T> fa;
    fa.xl = FX[lj * (A.nx + 1) + i];
    fa.xh = FX[lj * (A.nx + 1) + i + 1];
    fa.yl = FY[lj * A.nx + i];
    fa.yh = FY[(lj + 1) * A.nx + i];
    fa.zl = T(0);
    fa.zh = T(0);
    const T d = fsum(fa), m = MM[r];
    cx<T> nb = mk(T(0), T(0));
    if (i > 0) nb = axpy(fa.xl, Z[r - 1], nb);
    if (i < A.nx - 1) nb = axpy(fa.xh, Z[r + 1], nb);
    if (j > 0) nb = axpy(fa.yl, zrow(A, Z, lj - 1, i), nb);
    if (j < A.ny - 1) nb = axpy(fa.yh, zrow(A, Z, lj + 1, i), nb);
    const cx<T> Az = mk(fmaT(sft.re, m, d), mulT(sft.im, m)) * Z[r] - nb;
    return F[r] - Az;
  };

  // ---- down: smoothing and restriction on the banded levels
  for (int li = 0; li < P.nlev; ++li) {
    const ClLevel A = P.lev[li];
    for (int r = 0; r < 2; ++r) {
      sweep(A, 0, r == 0);
      sweep(A, 1, 0);
    }
    const int cnx = A.nx / 2;
    if (li + 1 < P.nlev) {
      const ClLevel B = P.lev[li + 1];
      cx<T>* FN = (cx<T>*)(csm + B.f);
      for (int t = tid; t < B.R * cnx; t += nt) {
        const int lJ = t / cnx, I = t - lJ * cnx;
        cx<T> acc = mk(T(0), T(0));
        for (int bb = 0; bb < 2; ++bb)
          for (int a = 0; a < 2; ++a) acc = acc + residual(A, 2 * I + a, 2 * lJ + bb);
        FN[t] = acc;
      }
      cl.sync();
    } else {
      // last banded level: residuals of the band, then CTA 0 restricts onto
      // the coarsest level and solves it with the dense inverse
      cx<T>* RS = (cx<T>*)(csm + P.rs);
      for (int t = tid; t < A.R * A.nx; t += nt) {
        const int lj = t / A.nx, i = t - lj * A.nx;
        RS[t] = residual(A, i, lj);
      }
      cl.sync();
      if (b == 0) {
        cx<T>* FC = (cx<T>*)(csm + P.fC);
        cx<T>* ZC = (cx<T>*)(csm + P.zC);
        for (int t = tid; t < P.nc; t += nt) {
          const int J = t / P.ncx, I = t - J * P.ncx;
          cx<T> acc = mk(T(0), T(0));
          for (int bb = 0; bb < 2; ++bb)
            for (int a = 0; a < 2; ++a) {
              const int j = 2 * J + bb, i = 2 * I + a;
              const int owner = j / A.R, lj = j - owner * A.R;
              acc = acc + cl.map_shared_rank(RS, owner)[lj * A.nx + i];
            }
          FC[t] = acc;
        }
        __syncthreads();
        const cx<T>* AI = (const cx<T>*)(csm + P.ainv);
        for (int rr = tid; rr < P.nc; rr += nt) {
          cx<T> acc = mk(T(0), T(0));
          const cx<T>* row = AI + (int64_t)rr * P.nc;
          for (int l = 0; l < P.nc; ++l) acc = acc + row[l] * FC[l];
          ZC[rr] = acc;
        }
      }
      cl.sync();
    }
  }

  // ---- up: prolongation and smoothing
  for (int li = P.nlev - 1; li >= 0; --li) {
    const ClLevel A = P.lev[li];
    cx<T>* Z = (cx<T>*)(csm + A.z);
    if (li + 1 < P.nlev) {
      const ClLevel B = P.lev[li + 1];
      cx<T>* ZB = (cx<T>*)(csm + B.z);
      auto get = [&](int X, int Y, int) -> cx<T> { return zrow(B, ZB, Y - b * B.R, X); };
      for (int t = tid; t < A.R * A.nx; t += nt) {
        const int lj = t / A.nx, i = t - lj * A.nx;
        Z[t] = Z[t] + prolong_value_at<T>(Cell{i, b * A.R + lj, 0}, 2, 2, 1, B.nx, B.ny, 1, P.mask, get);
      }
    } else {
      const cx<T>* ZC = cl.map_shared_rank((cx<T>*)(csm + P.zC), 0);
      auto get = [&](int X, int Y, int) -> cx<T> { return ZC[Y * P.ncx + X]; };
      for (int t = tid; t < A.R * A.nx; t += nt) {
        const int lj = t / A.nx, i = t - lj * A.nx;
        Z[t] = Z[t] + prolong_value_at<T>(Cell{i, b * A.R + lj, 0}, 2, 2, 1, P.ncx, P.ncy, 1, P.mask, get);
      }
    }
    cl.sync();
    for (int r = 0; r < 2; ++r) {
      sweep(A, 1, 0);
      sweep(A, 0, 0);
    }
  }
  {
    const ClLevel A = P.lev[0];
    const cx<T>* Z = (const cx<T>*)(csm + A.z);
    cx<T>* zo = P.z_out + slot * P.vs + (int64_t)b * A.R * A.nx;
    for (int q = tid; q < A.R * A.nx; q += nt) zo[q] = Z[q];
  }
}

// ------------------------------------------------------------------ host
template <typename T>
void launch_cluster_blob(const std::vector<LevelHost>& Ls, int l0, const ClusterParams<T>& P, const cx<T>* const* invd,
                         const cx<T>* Ainv, int ntau, unsigned char* blob, cudaStream_t s) {
  ClBlobArgs<T> A{};
  A.nlev = P.nlev;
  for (int i = 0; i < P.nlev; ++i) {
    const LevelHost& L = Ls[l0 + i];
    T* const* d = sizeof(T) == 8 ? (T* const*)L.d64 : (T* const*)L.d32;
    A.fx[i] = d[0];
    A.fy[i] = d[1];
    A.mm[i] = d[3];
    A.id[i] = invd[l0 + i];
    A.n[i] = L.n;
  }
  A.ainv = Ainv;
  k_cluster_blob<T><<<dim3(CL_SIZE, ntau), 256, 0, s>>>(P, A, blob);
}

template <typename T>
void cluster_prepare(size_t smem_bytes) {
  cudaFuncSetAttribute(k_cluster_vcycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

template <typename T>
bool cluster_launchable(size_t smem_bytes) {
  cluster_prepare<T>(smem_bytes);
  cudaLaunchConfig_t cfg = {};  // the cluster shape is the kernel's compile-time one
  cfg.gridDim = dim3(CL_SIZE);
  cfg.blockDim = dim3(CL_THREADS);
  cfg.dynamicSmemBytes = smem_bytes;
  int clusters = 0;
  cudaError_t e = cudaOccupancyMaxActiveClusters(&clusters, k_cluster_vcycle<T>, &cfg);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters > 0;
}

template <typename T>
void launch_cluster_vcycle(const ClusterParams<T>& P, size_t smem_bytes, const SlotState* st, int nslot,
                           cudaStream_t s) {
  k_cluster_vcycle<T><<<CL_SIZE * nslot, CL_THREADS, smem_bytes, s>>>(P, st);
}

#define CL_INST(T)                                                                                          \
  template bool cluster_layout<T>(const std::vector<LevelHost>&, int, ClusterParams<T>*, size_t*);          \
  template void launch_cluster_blob<T>(const std::vector<LevelHost>&, int, const ClusterParams<T>&,          \
                                       const cx<T>* const*, const cx<T>*, int, unsigned char*, cudaStream_t); \
  template void cluster_prepare<T>(size_t);                                                                 \
  template bool cluster_launchable<T>(size_t);                                                              \
  template void launch_cluster_vcycle<T>(const ClusterParams<T>&, size_t, const SlotState*, int, cudaStream_t);

CL_INST(double)
CL_INST(float)

}  // namespace fks
