// Device helpers for the cell-centred 2d+1-point operator, shared by the grid
// and Krylov kernels.
#pragma once
#include "common.cuh"

namespace fks {

// --------------------------------------------------------------------- indexing
struct Cell {
  int i, j, k;
};

__device__ __forceinline__ Cell cell_of(int64_t c, int nx, int ny) {
  Cell r;
  r.i = (int)(c % nx);
  int64_t q = c / nx;
  r.j = (int)(q % ny);
  r.k = (int)(q / ny);
  return r;
}

template <typename T>
struct Faces {
  T xl, xh, yl, yh, zl, zh;
};

template <typename T>
__device__ __forceinline__ Faces<T> faces_at(const LevelView<T>& L, Cell p) {
  Faces<T> f;
  int64_t rx = ((int64_t)p.k * L.ny + p.j) * (L.nx + 1) + p.i;
  f.xl = L.fx[rx];
  f.xh = L.fx[rx + 1];
  int64_t ry = ((int64_t)p.k * (L.ny + 1) + p.j) * L.nx + p.i;
  f.yl = L.fy[ry];
  f.yh = L.fy[ry + L.nx];
  if (L.nz > 1) {
    int64_t rz = ((int64_t)p.k * L.ny + p.j) * L.nx + p.i;
    f.zl = L.fz[rz];
    f.zh = L.fz[rz + (int64_t)L.nx * L.ny];
  } else {
    f.zl = T(0);
    f.zh = T(0);
  }
  return f;
}

template <typename T>
__device__ __forceinline__ T fsum(const Faces<T>& f) {
  return ((f.xl + f.xh) + (f.yl + f.yh)) + (f.zl + f.zh);
}

// sum over existing neighbours of t_face * x_nb
template <typename T>
__device__ __forceinline__ cx<T> nb_sum(const LevelView<T>& L, const Faces<T>& f, Cell p, int64_t c,
                                        const cx<T>* __restrict__ x) {
  cx<T> s = mk(T(0), T(0));
  int64_t sxy = (int64_t)L.nx * L.ny;
  if (p.i > 0) s = s + f.xl * x[c - 1];
  if (p.i < L.nx - 1) s = s + f.xh * x[c + 1];
  if (p.j > 0) s = s + f.yl * x[c - L.nx];
  if (p.j < L.ny - 1) s = s + f.yh * x[c + L.nx];
  if (L.nz > 1) {
    if (p.k > 0) s = s + f.zl * x[c - sxy];
    if (p.k < L.nz - 1) s = s + f.zh * x[c + sxy];
  }
  return s;
}

template <typename T>
__device__ __forceinline__ cx<T> apply_at(const LevelView<T>& L, Cell p, int64_t c, cx<T> s,
                                          const cx<T>* __restrict__ x) {
  Faces<T> f = faces_at(L, p);
  T d = fsum(f);
  T m = L.mm[c];
  cx<T> diag = mk(d + s.re * m, s.im * m);
  return diag * x[c] - nb_sum(L, f, p, c, x);
}

}  // namespace fks
