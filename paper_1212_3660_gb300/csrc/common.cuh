// Internal types shared by the kernels and the host engine.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <string>
#include <vector>

namespace fks {

// ---------------------------------------------------------------- complex
template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

// Rounding is pinned with explicit intrinsics (no compiler FMA contraction
// choices), so that every kernel that computes the same update gets the same bits.
template <typename T>
__host__ __device__ __forceinline__ T fmaT(T a, T b, T c) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(T) == 8) return __fma_rn(a, b, c); else return __fmaf_rn(a, b, c);
#else
  return std::fma(a, b, c);
#endif
}
template <typename T>
__host__ __device__ __forceinline__ T mulT(T a, T b) {
#ifdef __CUDA_ARCH__
  if constexpr (sizeof(T) == 8) return __dmul_rn(a, b); else return __fmul_rn(a, b);
#else
  return a * b;
#endif
}

template <typename T>
__host__ __device__ __forceinline__ cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.re + b.re, a.im + b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.re - b.re, a.im - b.im); }
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(fmaT(a.re, b.re, -mulT(a.im, b.im)), fmaT(a.re, b.im, mulT(a.im, b.re)));
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk(mulT(s, a.re), mulT(s, a.im)); }
// acc + s * x (real s)
template <typename T>
__host__ __device__ __forceinline__ cx<T> axpy(T s, cx<T> x, cx<T> acc) {
  return mk(fmaT(s, x.re, acc.re), fmaT(s, x.im, acc.im));
}
template <typename T>
__host__ __device__ __forceinline__ cx<T> conj(cx<T> a) { return mk(a.re, -a.im); }
template <typename T>
__host__ __device__ __forceinline__ T abs2(cx<T> a) { return fmaT(a.re, a.re, mulT(a.im, a.im)); }
// conj(a) * b
template <typename T>
__host__ __device__ __forceinline__ cx<T> cdot(cx<T> a, cx<T> b) {
  return mk(fmaT(a.re, b.re, mulT(a.im, b.im)), fmaT(a.re, b.im, -mulT(a.im, b.re)));
}
template <typename To, typename Ti>
__host__ __device__ __forceinline__ cx<To> cvt(cx<Ti> a) { return mk((To)a.re, (To)a.im); }

typedef cx<double> z64;
typedef cx<float> z32;

// ---------------------------------------------------------------- grid level
// Coefficients of one multigrid level in precision T. Faces are stored for the
// whole closed grid: fx has (nx+1) entries per x-row, fx[row*(nx+1) + i] being the
// transmissibility of the face between cells i-1 and i (i = 0 and i = nx are the
// boundary faces: 2 K A / h on a zero-head face, 0 on a no-flow face); likewise
// fy with (ny+1) rows per plane and fz with (nz+1) planes. mm is the diagonal of M.
// The diagonal of K at a cell is the sum of its 2d faces.
// C is the storage type of the coefficients (T itself, or bf16 / float
// copies read into T arithmetic); kd is always T.
template <typename T, typename C = T>
struct LevelView {
  int nx, ny, nz;
  int64_t n;
  const C* fx;
  const C* fy;
  const C* fz;  // unused when nz == 1
  const C* mm;
  const T* kd;  // diagonal of K (sum of the cell's faces), when precomputed; else null
};

// coefficient i of a C array in arithmetic type T
template <typename T, typename C>
__host__ __device__ __forceinline__ T ldc(const C* p, int64_t i) {
  if constexpr (sizeof(C) == 2) return (T)__bfloat162float(p[i]);
  else return (T)p[i];
}

// ---------------------------------------------------------------- launch overlap
// Programmatic dependent launch: a kernel launched by launch_pdl may be
// scheduled while its predecessor in the stream is still running. It waits in
// pdl_enter for the predecessor's completion (and the visibility of its
// writes) before it touches global memory, then lets its own successor begin
// launching. Without the launch attribute both instructions are no-ops.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// process-wide switch (on by default; fks_set_pdl)
inline int& pdl_flag() {
  static int on = 1;
  return on;
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_flag() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

constexpr int MAX_LEVELS = 16;
constexpr int MAX_COARSE = 1024;
constexpr int MAX_TAU = 16;
constexpr int MAX_M = 128;

struct LevelHost {
  int nx, ny, nz;
  int rx, ry, rz;     // ratio to the NEXT coarser level (1 or 2); 1,1,1 on the coarsest
  int64_t n;
  double h[3];
  double* d64[4];     // fx, fy, fz, mm (device)
  float* d32[4];      // fp32 copies (device)
  double* kd64;       // diagonal of K in fp64 (finest level only; else null)
  // the bf16-smoother option: the coefficients rounded to bf16 (d16), and the
  // same rounded values as fp32 (d32b) for the kernels that read fp32
  __nv_bfloat16* d16[4];
  float* d32b[4];
};

// A view of the level's coefficients stored as C (double: d64, float: d32,
// bf16: d16), read in arithmetic type T; no precomputed diagonal.
template <typename T, typename C>
inline LevelView<T, C> view_as(const LevelHost& L) {
  LevelView<T, C> v;
  v.nx = L.nx; v.ny = L.ny; v.nz = L.nz; v.n = L.n;
  C* const* a;
  if constexpr (sizeof(C) == 8) a = (C* const*)L.d64;
  else if constexpr (sizeof(C) == 4) a = (C* const*)L.d32;
  else a = (C* const*)L.d16;
  v.fx = a[0]; v.fy = a[1]; v.fz = a[2]; v.mm = a[3];
  v.kd = nullptr;
  return v;
}

template <typename T>
inline LevelView<T> view(const LevelHost& L) {
  LevelView<T> v;
  v.nx = L.nx; v.ny = L.ny; v.nz = L.nz; v.n = L.n;
  T* const* a;
  if constexpr (sizeof(T) == 8) a = (T* const*)L.d64; else a = (T* const*)L.d32;
  v.fx = a[0]; v.fy = a[1]; v.fz = a[2]; v.mm = a[3];
  if constexpr (sizeof(T) == 8) v.kd = (const T*)L.kd64; else v.kd = nullptr;
  return v;
}

inline int64_t face_count(const LevelHost& L, int a) {
  return a == 0 ? (int64_t)(L.nx + 1) * L.ny * L.nz
       : a == 1 ? (int64_t)L.nx * (L.ny + 1) * L.nz
                : (int64_t)L.nx * L.ny * (L.nz + 1);
}

// ---------------------------------------------------------------- per-source state
// Small per-source (slot) state kept in device memory so that every kernel of a
// step can read it without host involvement.
struct SlotState {
  double beta;      // ||b||
  double vnorm2;    // ||v_k||^2
  double pnorm2;    // ||v_k - (K + tau_k M) z||^2 of the current inner iterate
  double w0norm2;   // ||M z_k||^2 (scale of the breakdown test)
  int k;            // current step, 1-based (set when the step starts)
  int tau;          // index of tau_bar for step k
  int cycles;       // inner cycles done in this step
  int inner_done;   // inner solve of this step finished
  int active;       // source still iterating
  int live;         // shifts not yet frozen
  int breakdown;    // h_{k+1,k} vanished at step k
  int inner_capped; // some inner solve hit its cycle cap
  double rmax;      // largest relative residual estimate of the live shifts after the last step (1 at start)
  unsigned long long rmax_next;  // the same for the step in progress (bits of a non-negative double, atomic max)
};

constexpr double RELAX_EPS_MAX = 1e-3;  // cap on a relaxed inner tolerance

// Inner tolerance of the current step: eps, or with relax > 0 the relaxed
// min(RELAX_EPS_MAX, max(eps, relax * tol / rmax)) (Section 4's closing remark).
__host__ __device__ inline double inner_eps(double eps, double relax, double tol, double rmax) {
  if (!(relax > 0.0)) return eps;
  double e = rmax > 0.0 ? relax * tol / rmax : RELAX_EPS_MAX;
  return fmin(RELAX_EPS_MAX, fmax(eps, e));
}

// Fixed-order block reduction of one double (blockDim.x a multiple of 32, at
// most 1024); the result is valid in thread 0. Deterministic for a given
// blockDim, so the same inputs always give the same bits.
__device__ __forceinline__ double block_sum(double v, double* scratch32) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) scratch32[w] = v;
  __syncthreads();
  int nw = blockDim.x >> 5;
  v = threadIdx.x < nw ? scratch32[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  return v;
}

// error reporting
void set_error(const std::string& msg);
const char* get_error();

}  // namespace fks
