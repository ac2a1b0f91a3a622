// The lower multigrid levels of a V-cycle in one cooperative launch (see
// coop.cuh). Every phase is a grid-stride loop over (source, cell) work items,
// followed by a grid-wide barrier; each cell's update is the one the per-level
// kernels and the tail kernel compute (gs_value, restrict_value,
// prolong_value and the coarsest product in the same order), so the results
// are bitwise the same whichever runs.
#include <cooperative_groups.h>

#include <algorithm>
#include <atomic>

#include "coop.cuh"
#include "stencil.cuh"

namespace cg = cooperative_groups;

namespace fks {

constexpr int COOP_THREADS = 256;

__device__ __forceinline__ bool coop_running(const SlotState* st, int slot) {
  return st[slot].active && !st[slot].inner_done;
}

template <typename T>
__global__ void __launch_bounds__(COOP_THREADS) k_coop_vcycle(CoopParams<T> P, const SlotState* __restrict__ st) {
  cg::grid_group grid = cg::this_grid();
  const int64_t g0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  const int ns = P.nslot;

  // one red-black half sweep of level l on every running source
  auto sweep = [&](int l, int color, int zs) {
    const LevelView<T>& L = P.L[l];
    const int64_t work = (int64_t)((L.nx + 1) >> 1) * L.ny * L.nz;
    for (int64_t w = g0; w < work * ns; w += gs) {
      const int slot = (int)(w / work);
      if (!coop_running(st, slot)) continue;
      Cell p;
      int c;
      if (!color_cell(L.nx, L.ny, L.nz, color, (int)(w - slot * work), &p, &c)) continue;
      cx<T>* F = P.f[l] + (int64_t)slot * L.n;
      cx<T>* Z = P.z[l] + (int64_t)slot * L.n;
      const cx<T>* ID = P.invd[l] + (int64_t)st[slot].tau * L.n;
      Z[c] = gs_value(L, p, c, ID[c], F, Z, zs);
    }
    grid.sync();
  };

  for (int l = 0; l + 1 < P.nlev; ++l) {
    for (int r = 0; r < 2; ++r) {
      sweep(l, 0, r == 0);
      sweep(l, 1, 0);
    }
    const LevelView<T>& A = P.L[l];
    const LevelView<T>& B = P.L[l + 1];
    for (int64_t w = g0; w < B.n * ns; w += gs) {
      const int slot = (int)(w / B.n);
      if (!coop_running(st, slot)) continue;
      const int C = (int)(w - slot * B.n);
      const Cell pc = cell_of(C, B.nx, B.ny);
      const cx<T> sft = cvt<T>(P.taus[st[slot].tau]);
      P.f[l + 1][(int64_t)slot * B.n + C] =
          restrict_value(A, P.rx[l], P.ry[l], P.rz[l], pc.i, pc.j, pc.k, sft, P.f[l] + (int64_t)slot * A.n,
                         P.z[l] + (int64_t)slot * A.n);
    }
    grid.sync();
  }
  {
    // coarsest level: z = A^{-1} f
    const int l = P.nlev - 1;
    for (int64_t w = g0; w < (int64_t)P.nc * ns; w += gs) {
      const int slot = (int)(w / P.nc);
      if (!coop_running(st, slot)) continue;
      const int r = (int)(w - (int64_t)slot * P.nc);
      const cx<T>* row = P.Ainv + ((int64_t)st[slot].tau * P.nc + r) * P.nc;
      const cx<T>* F = P.f[l] + (int64_t)slot * P.nc;
      cx<T> acc = mk(T(0), T(0));
      for (int q = 0; q < P.nc; ++q) acc = acc + row[q] * F[q];
      P.z[l][(int64_t)slot * P.nc + r] = acc;
    }
    grid.sync();
  }
  for (int l = P.nlev - 2; l >= 0; --l) {
    const LevelView<T>& A = P.L[l];
    const LevelView<T>& B = P.L[l + 1];
    for (int64_t w = g0; w < A.n * ns; w += gs) {
      const int slot = (int)(w / A.n);
      if (!coop_running(st, slot)) continue;
      const int c = (int)(w - slot * A.n);
      const Cell p = cell_of(c, A.nx, A.ny);
      cx<T>* Z = P.z[l] + (int64_t)slot * A.n;
      Z[c] = Z[c] + prolong_value(p, P.rx[l], P.ry[l], P.rz[l], B.nx, B.ny, B.nz, P.mask,
                                  P.z[l + 1] + (int64_t)slot * B.n);
    }
    grid.sync();
    for (int r = 0; r < 2; ++r) {
      sweep(l, 1, 0);
      sweep(l, 0, 0);
    }
  }
}

// resident blocks per device, cached (count + 1; 0 = not yet known)
constexpr int COOPV_MAX_DEVICES = 64;
static std::atomic<int> g_coopv_resident[2][COOPV_MAX_DEVICES];

template <typename T>
int coop_capacity_vcycle() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= COOPV_MAX_DEVICES) {
    cudaGetLastError();
    return 0;
  }
  const int which = sizeof(T) == 8 ? 0 : 1;
  const int r = g_coopv_resident[which][dev].load(std::memory_order_relaxed);
  if (r > 0) return r - 1;
  int sms = 0, per = 0, coop = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
  if (!coop || cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_coop_vcycle<T>, COOP_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    per = 0;
  }
  g_coopv_resident[which][dev].store(per * sms + 1, std::memory_order_relaxed);
  return per * sms;
}

template <typename T>
bool launch_coop_vcycle(const CoopParams<T>& P, const SlotState* st, int blocks, cudaStream_t s) {
  const int cap = coop_capacity_vcycle<T>();
  if (cap <= 0 || st == nullptr) return false;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::max(1, std::min(blocks, cap)));
  cfg.blockDim = dim3(COOP_THREADS);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaLaunchKernelEx(&cfg, k_coop_vcycle<T>, P, st) == cudaSuccess) return true;
  cudaGetLastError();
  return false;
}

#define FKS_COOP_INST(T)                                                                              \
  template int coop_capacity_vcycle<T>();                                                             \
  template bool launch_coop_vcycle<T>(const CoopParams<T>&, const SlotState*, int, cudaStream_t);
FKS_COOP_INST(float)
FKS_COOP_INST(double)

}  // namespace fks
