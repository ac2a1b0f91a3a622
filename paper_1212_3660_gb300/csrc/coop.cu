// The lower multigrid levels of a V-cycle in one launch (see coop.cuh), in one
// of two forms: one thread-block cluster per source (its CTAs share the
// source's cells; cluster barriers between phases), or one cooperative grid
// over all sources (grid-wide barriers). Every phase is a strided loop over
// (source, cell) work items followed by the barrier; each cell's update is the
// one the per-level kernels and the tail kernel compute (gs_value,
// restrict_value, prolong_value and the coarsest product in the same order), so
// the results are bitwise the same whichever runs.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "coop.cuh"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace fks {

constexpr int COOP_THREADS = 256;
constexpr int64_t COOP_CLUSTER_MAX_CELLS = 65536;  // largest level of the per-source cluster form

__device__ __forceinline__ bool coop_running(const SlotState* st, int slot) {
  return st[slot].active && !st[slot].inner_done;
}

template <typename T, bool CLUSTER>
__global__ void __launch_bounds__(COOP_THREADS) k_coop_vcycle(CoopParams<T> P, const SlotState* __restrict__ st) {
  // CLUSTER: the cluster of blockIdx.x / cluster size works on that source alone
  int64_t g0, gs;
  int s0, ns;
  if constexpr (CLUSTER) {
    cg::cluster_group cl = cg::this_cluster();
    g0 = (int64_t)cl.block_rank() * blockDim.x + threadIdx.x;
    gs = (int64_t)cl.num_blocks() * blockDim.x;
    s0 = (int)(blockIdx.x / cl.num_blocks());
    ns = 1;
  } else {
    g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    gs = (int64_t)gridDim.x * blockDim.x;
    s0 = 0;
    ns = P.nslot;
  }
  auto barrier = [&]() {
    if constexpr (CLUSTER) cg::this_cluster().sync();
    else cg::this_grid().sync();
  };

  // one red-black half sweep of level l on every running source
  auto sweep = [&](int l, int color, int zs) {
    const LevelView<T>& L = P.L[l];
    const int64_t work = (int64_t)((L.nx + 1) >> 1) * L.ny * L.nz;
    for (int64_t w = g0; w < work * ns; w += gs) {
      const int slot = s0 + (int)(w / work);
      if (!coop_running(st, slot)) continue;
      Cell p;
      int c;
      if (!color_cell(L.nx, L.ny, L.nz, color, (int)(w - (slot - s0) * work), &p, &c)) continue;
      cx<T>* F = P.f[l] + (int64_t)slot * L.n;
      cx<T>* Z = P.z[l] + (int64_t)slot * L.n;
      const cx<T>* ID = P.invd[l] + (int64_t)st[slot].tau * L.n;
      Z[c] = gs_value(L, p, c, ID[c], F, Z, zs);
    }
    barrier();
  };

  for (int l = 0; l + 1 < P.nlev; ++l) {
    for (int r = 0; r < 2; ++r) {
      sweep(l, 0, r == 0);
      sweep(l, 1, 0);
    }
    const LevelView<T>& A = P.L[l];
    const LevelView<T>& B = P.L[l + 1];
    for (int64_t w = g0; w < B.n * ns; w += gs) {
      const int slot = s0 + (int)(w / B.n);
      if (!coop_running(st, slot)) continue;
      const int C = (int)(w - (slot - s0) * B.n);
      const Cell pc = cell_of(C, B.nx, B.ny);
      const cx<T> sft = cvt<T>(P.taus[st[slot].tau]);
      P.f[l + 1][(int64_t)slot * B.n + C] =
          restrict_value(A, P.rx[l], P.ry[l], P.rz[l], pc.i, pc.j, pc.k, sft, P.f[l] + (int64_t)slot * A.n,
                         P.z[l] + (int64_t)slot * A.n);
    }
    barrier();
  }
  {
    // coarsest level: z = A^{-1} f
    const int l = P.nlev - 1;
    for (int64_t w = g0; w < (int64_t)P.nc * ns; w += gs) {
      const int slot = s0 + (int)(w / P.nc);
      if (!coop_running(st, slot)) continue;
      const int r = (int)(w - (int64_t)(slot - s0) * P.nc);
      const cx<T>* row = P.Ainv + ((int64_t)st[slot].tau * P.nc + r) * P.nc;
      const cx<T>* F = P.f[l] + (int64_t)slot * P.nc;
      cx<T> acc = mk(T(0), T(0));
      for (int q = 0; q < P.nc; ++q) acc = acc + row[q] * F[q];
      P.z[l][(int64_t)slot * P.nc + r] = acc;
    }
    barrier();
  }
  for (int l = P.nlev - 2; l >= 0; --l) {
    const LevelView<T>& A = P.L[l];
    const LevelView<T>& B = P.L[l + 1];
    for (int64_t w = g0; w < A.n * ns; w += gs) {
      const int slot = s0 + (int)(w / A.n);
      if (!coop_running(st, slot)) continue;
      const int c = (int)(w - (slot - s0) * A.n);
      const Cell p = cell_of(c, A.nx, A.ny);
      cx<T>* Z = P.z[l] + (int64_t)slot * A.n;
      Z[c] = Z[c] + prolong_value(p, P.rx[l], P.ry[l], P.rz[l], B.nx, B.ny, B.nz, P.mask,
                                  P.z[l + 1] + (int64_t)slot * B.n);
    }
    barrier();
    for (int r = 0; r < 2; ++r) {
      sweep(l, 1, 0);
      sweep(l, 0, 0);
    }
  }
}

// per device, cached (value + 1; 0 = not yet known): resident blocks of the
// grid-wide form, and the cluster size of the per-source form (16 or 8; 0 if
// no cluster of either size can be resident)
constexpr int COOPV_MAX_DEVICES = 64;
static std::atomic<int> g_coopv_resident[2][COOPV_MAX_DEVICES];
static std::atomic<int> g_coopv_cluster[2][COOPV_MAX_DEVICES];

static int coopv_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= COOPV_MAX_DEVICES) {
    cudaGetLastError();
    return -1;
  }
  return dev;
}

template <typename T>
static int coop_grid_capacity() {
  const int dev = coopv_device();
  if (dev < 0) return 0;
  const int which = sizeof(T) == 8 ? 0 : 1;
  const int r = g_coopv_resident[which][dev].load(std::memory_order_relaxed);
  if (r > 0) return r - 1;
  int sms = 0, per = 0, coop = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coop_vcycle<T, false>, COOP_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  g_coopv_resident[which][dev].store(per * sms + 1, std::memory_order_relaxed);
  return per * sms;
}

template <typename T>
static int coop_cluster_size() {
  const int dev = coopv_device();
  if (dev < 0) return 0;
  const int which = sizeof(T) == 8 ? 0 : 1;
  const int r = g_coopv_cluster[which][dev].load(std::memory_order_relaxed);
  if (r > 0) return r - 1;
  int pick = 0;
  for (int cs : {16, 8}) {
    if (cudaFuncSetAttribute(k_coop_vcycle<T, true>, cudaFuncAttributeNonPortableClusterSizeAllowed, cs > 8 ? 1 : 0) !=
        cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(COOP_THREADS);
    cudaLaunchAttribute a[1];
    a[0].id = cudaLaunchAttributeClusterDimension;
    a[0].val.clusterDim.x = cs;
    a[0].val.clusterDim.y = 1;
    a[0].val.clusterDim.z = 1;
    cfg.attrs = a;
    cfg.numAttrs = 1;
    int ncl = 0;
    if (cudaOccupancyMaxActiveClusters(&ncl, k_coop_vcycle<T, true>, &cfg) == cudaSuccess && ncl > 0) {
      pick = cs;
      break;
    }
    cudaGetLastError();
  }
  g_coopv_cluster[which][dev].store(pick + 1, std::memory_order_relaxed);
  return pick;
}

template <typename T>
int coop_capacity_vcycle() {
  return coop_grid_capacity<T>() > 0 ? 1 : coop_cluster_size<T>();
}

template <typename T>
bool launch_coop_vcycle(const CoopParams<T>& P, const SlotState* st, int blocks, cudaStream_t s) {
  if (st == nullptr) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.blockDim = dim3(COOP_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // one cluster per source while the largest level is small (its CTAs then
  // have little work per phase and a cluster barrier is the cheaper one); else
  // the grid-wide form over every SM
  int64_t most = 0;
  for (int l = 0; l < P.nlev; ++l) most = std::max<int64_t>(most, P.L[l].n);
  const int cs = coop_cluster_size<T>(), cap = coop_grid_capacity<T>();
  if (cs > 0 && (most <= COOP_CLUSTER_MAX_CELLS || cap <= 0)) {
    // one cluster per source
    cfg.gridDim = dim3(cs * P.nslot);
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    if (cudaLaunchKernelEx(&cfg, k_coop_vcycle<T, true>, P, st) == cudaSuccess) return true;
    cudaGetLastError();
    return false;
  }
  if (cap <= 0) return false;
  cfg.gridDim = dim3(std::max(1, std::min(blocks, cap)));
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  if (cudaLaunchKernelEx(&cfg, k_coop_vcycle<T, false>, P, st) == cudaSuccess) return true;
  cudaGetLastError();
  return false;
}

#define FKS_COOP_INST(T)                                                                              \
  template int coop_capacity_vcycle<T>();                                                             \
  template bool launch_coop_vcycle<T>(const CoopParams<T>&, const SlotState*, int, cudaStream_t);
FKS_COOP_INST(float)
FKS_COOP_INST(double)

}  // namespace fks
