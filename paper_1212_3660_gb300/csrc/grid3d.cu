// Fused 3D multigrid level kernels (the inexact inner solve of Section 4,
// Eq. zmmoditer, on a 3D grid coarsened by 2 in every axis).
//
// One kernel per half of the V-cycle on a level, over tiles of TX x TY cells
// in the x-y plane and a chunk of planes in z. A block marches through its
// planes ("2.5D"): at march step p it loads plane p and runs the first half
// sweep there, the second half sweep on plane p - 1, the third on p - 2, the
// fourth on p - 3, and the residual (pre) or the output (post) of plane p - 5.
// Red-black half sweeps only read the other colour, so this wavefront reads
// every neighbour in the version the per-sweep kernels would see (the
// ordering is argued beside k_pre3d). In x and y the tile carries a halo of
// FH = 4 cells that is recomputed, shrinking by one cell per half sweep, as in
// the 2D fused kernels; in z the chunk is widened by 4 planes on each side the
// same way. Values of plane q live in ring slot q mod R of shared memory.
// Every cell update repeats the per-level kernels' arithmetic in the same
// order, so the results are bitwise those of k_gs / k_residual_restrict /
// k_prolong_add / k_correct.
//   pre : z = four half sweeps from z = 0 (red, black, red, black); write z;
//         coarse f = sum over the 8 children of (f - A z)
//   post: z += P z_coarse; four half sweeps (black, red, black, red); write z
//         (or, on the finest level, add it to the outer iterate z_k)
#include <algorithm>

#include "grid.cuh"
#include "stencil.cuh"

namespace fks {

constexpr int R3Z = 7;       // planes of z in the ring
constexpr int R3F = 6;       // planes of f in the ring

// Tile geometry and block size: one thread per interior cell (the residual and
// the output take one cell each) and at least one per cell of a half sweep on
// the region shrunk by one cell, so every phase but the plane load gives each
// thread at most one cell; the plane load takes LOADS cells per thread.
template <int TX, int TY>
struct Tile3 {
  static constexpr int RX = TX + 2 * FH, RY = TY + 2 * FH, P = RX * RY;
  static constexpr int NT = TX * TY >= 512 ? 512 : (TX * TY >= 256 ? 256 : 128);
  static constexpr int LOADS = (P + NT - 1) / NT;
  static_assert(TX * TY <= NT && ((RX - 1) / 2) * (RY - 2) <= NT, "one cell per thread per phase");
  static_assert((TX * TY) % 32 == 0, "the residual combines children within whole warps");
};

__device__ __forceinline__ bool slot_running3(const SlotState* st, int slot) {
  return st == nullptr || (st[slot].active && !st[slot].inner_done);
}

// s + sum over existing neighbours of t_face * z_nb, in the order of nb_sum
// (x low, x high, y low, y high, z low, z high); Zq holds the cell's plane,
// Zm / Zp the planes below / above, r is the cell's index in the plane.
template <typename T, int RX>
__device__ __forceinline__ cx<T> nb_sum3(const LevelView<T>& L, const Faces<T>& f, int gx, int gy, int q, int r,
                                         const cx<T>* Zm, const cx<T>* Zq, const cx<T>* Zp, cx<T> s) {
  if (gx > 0) s = axpy(f.xl, Zq[r - 1], s);
  if (gx < L.nx - 1) s = axpy(f.xh, Zq[r + 1], s);
  if (gy > 0) s = axpy(f.yl, Zq[r - RX], s);
  if (gy < L.ny - 1) s = axpy(f.yh, Zq[r + RX], s);
  if (q > 0) s = axpy(f.zl, Zm[r], s);
  if (q < L.nz - 1) s = axpy(f.zh, Zp[r], s);
  return s;
}

__device__ __forceinline__ bool plane_in(int q, int lo, int hi, int nz) { return q >= lo && q < hi && q >= 0 && q < nz; }

// This thread's cell of a red-black half sweep of colour `color` on plane q
// over the tile region shrunk by `sh` cells, with its coefficients fetched
// ahead of the barrier that precedes the update (r < 0: no cell).
template <typename T>
struct SwCell {
  int r, gx, gy;
  Faces<T> fa;
  cx<T> id;
};

template <typename T, int TX, int TY>
__device__ __forceinline__ void sw_fetch(const LevelView<T>& L, const cx<T>* __restrict__ ID, int x0, int y0, int q,
                                         int color, int sh, bool on, SwCell<T>& S) {
  constexpr int RX = Tile3<TX, TY>::RX, RY = Tile3<TX, TY>::RY;
  S.r = -1;
  if (!on) return;
  const int w = RX - 2 * sh, hgt = RY - 2 * sh, wh = (w + 1) >> 1;
  const int it = threadIdx.x;
  if (it >= wh * hgt) return;
  const int yy = it / wh;
  const int ry = sh + yy, gy = y0 + ry;
  int rx0 = sh + 2 * (it - yy * wh), gx = x0 + rx0;
  if (((gx + gy + q) & 1) != color) { ++gx; ++rx0; }
  if (rx0 >= RX - sh || gx < 0 || gx >= L.nx || gy < 0 || gy >= L.ny) return;
  S.r = ry * RX + rx0;
  S.gx = gx;
  S.gy = gy;
  S.fa = faces_at(L, Cell{gx, gy, q});
  S.id = ID[((int64_t)q * L.ny + gy) * L.nx + gx];
}

// z_c = (f_c + sum_nb t z_nb) / (K_cc + tau M_cc) for the fetched cell
template <typename T, int TX, int TY>
__device__ __forceinline__ void sw_apply(const LevelView<T>& L, int q, const SwCell<T>& S, cx<T>* sZ,
                                         const cx<T>* sF) {
  constexpr int RX = Tile3<TX, TY>::RX, P = Tile3<TX, TY>::P;
  if (S.r < 0) return;
  cx<T>* Zq = sZ + (q % R3Z) * P;
  const cx<T>* Zm = sZ + ((q + R3Z - 1) % R3Z) * P;
  const cx<T>* Zp = sZ + ((q + 1) % R3Z) * P;
  const cx<T>* Fq = sF + (q % R3F) * P;
  const cx<T> rhs = nb_sum3<T, RX>(L, S.fa, S.gx, S.gy, q, S.r, Zm, Zq, Zp, Fq[S.r]);
  Zq[S.r] = S.id * rhs;
}

template <typename T>
__device__ __forceinline__ cx<T> shfl_cx(cx<T> v, int lane) {
  return mk(__shfl_sync(0xffffffffu, v.re, lane), __shfl_sync(0xffffffffu, v.im, lane));
}

// Ordering at march step p (phases separated by block barriers):
//   1: output of plane p - 4 (final: its black cells took their last sweep in
//      phase 4 of step p - 1), residual of plane p - 5 (reads z of p - 6 ..
//      p - 4, f of p - 5) and load of plane p with the first (red,
//      zero-start) half sweep there (writes ring slots of p, which hold p - 7
//      for z and p - 6 for f)
//   2: black half sweep on p - 1 (reads red of p - 2 .. p: first-sweep values;
//      red of p - 2 is updated only in phase 3)
//   3: red on p - 2 (reads black of p - 3 .. p - 1: second-sweep values;
//      black of p - 3 is updated only in phase 4)
//   4: black on p - 3 (reads red of p - 4 .. p - 2: third-sweep values, final)
// and the residual of plane q reads final values of q - 1 .. q + 1 (black of
// q + 1 became final at phase 4 of step q + 4). The coefficients of phases 2-4
// are fetched at the start of phase 1, so their latency overlaps it.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(Tile3<TX, TY>::NT) k_pre3d(LevelView<T> L, const SlotState* st,
                                                             const cx<T>* __restrict__ invd, const z64* taus,
                                                             const cx<T>* __restrict__ f, cx<T>* __restrict__ z,
                                                             int64_t vs, cx<T>* __restrict__ fc, int64_t vsc, int zc) {
  constexpr int RX = Tile3<TX, TY>::RX, P = Tile3<TX, TY>::P, NT = Tile3<TX, TY>::NT;
  constexpr int LOADS = Tile3<TX, TY>::LOADS;
  constexpr int CX = TX / 2;
  extern __shared__ __align__(16) unsigned char pre3_smem[];
  cx<T>* sZ = (cx<T>*)pre3_smem;
  cx<T>* sF = sZ + R3Z * P;
  cx<T>* sC = sF + R3F * P;
  const int slot = blockIdx.z;
  if (!slot_running3(st, slot)) return;
  const int tau = st[slot].tau;
  const cx<T> sft = cvt<T>(taus[tau]);
  const cx<T>* ID = invd + (int64_t)tau * L.n;
  const cx<T>* fs = f + slot * vs;
  cx<T>* zs = z + slot * vs;
  cx<T>* fcs = fc + slot * vsc;
  const int ntx = (L.nx + TX - 1) / TX;
  const int bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
  const int x0 = bx * TX - FH, y0 = by * TY - FH;
  const int z0 = blockIdx.y * zc, z1 = min(z0 + zc, L.nz);
  const int cnx = L.nx >> 1, cny = L.ny >> 1;
  const int tid = threadIdx.x;
  // this thread's interior cell (output) and child of a coarse cell (residual)
  const int ox = tid % TX, oy = tid / TX;
  const int ck = tid >> 2, cb = (tid >> 1) & 1, ca = tid & 1;
  const int cX = bx * CX + ck % CX, cY = by * (TY / 2) + ck / CX;
  const bool cvalid = tid < TX * TY && cX < cnx && cY < cny;
  const int cgx = 2 * cX + ca, cgy = 2 * cY + cb;
  const int cr = (cgy - y0) * RX + (cgx - x0);
  const int pfirst = max(z0 - FH, 0), plast = z1 + FH;
  for (int p = pfirst; p <= plast; ++p) {
    SwCell<T> s1, s2, s3;
    sw_fetch<T, TX, TY>(L, ID, x0, y0, p - 1, 1, 1, plane_in(p - 1, z0 - 3, z1 + 3, L.nz), s1);
    sw_fetch<T, TX, TY>(L, ID, x0, y0, p - 2, 0, 2, plane_in(p - 2, z0 - 2, z1 + 2, L.nz), s2);
    sw_fetch<T, TX, TY>(L, ID, x0, y0, p - 3, 1, 3, plane_in(p - 3, z0 - 1, z1 + 1, L.nz), s3);
    // phase 1a: load plane p (all loads first) ...
    const bool load = plane_in(p, z0 - FH, z1 + FH, L.nz);
    cx<T> fv[LOADS], iv[LOADS];
    bool red[LOADS];
#pragma unroll
    for (int u = 0; u < LOADS; ++u) {
      const int it = tid + u * NT;
      const int ry = it / RX, rx = it - ry * RX;
      const int gx = x0 + rx, gy = y0 + ry;
      const bool in = load && it < P && gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny;
      const int64_t c = ((int64_t)p * L.ny + gy) * L.nx + gx;
      red[u] = in && ((gx + gy + p) & 1) == 0;
      fv[u] = in ? fs[c] : mk(T(0), T(0));
      iv[u] = red[u] ? ID[c] : mk(T(0), T(0));
    }
    // phase 1b: the smoothed interior of plane p - 4 (both colours final) to z
    const int qo = p - 4;
    if (qo >= z0 && qo < z1 && tid < TX * TY) {
      const int gx = x0 + FH + ox, gy = y0 + FH + oy;
      if (gx < L.nx && gy < L.ny)
        zs[((int64_t)qo * L.ny + gy) * L.nx + gx] = sZ[(qo % R3Z) * P + (oy + FH) * RX + ox + FH];
    }
    // phase 1c: residual of plane q = p - 5, one child cell per thread, summed
    // into its coarse cell in the per-level kernel's child order (b, then a)
    const int qr = p - 5;
    if (qr >= z0 && qr < z1 && tid < TX * TY) {
      cx<T> v = mk(T(0), T(0));
      if (cvalid) {
        const cx<T>* Zq = sZ + (qr % R3Z) * P;
        const cx<T>* Zm = sZ + ((qr + R3Z - 1) % R3Z) * P;
        const cx<T>* Zp = sZ + ((qr + 1) % R3Z) * P;
        const int64_t c = ((int64_t)qr * L.ny + cgy) * L.nx + cgx;
        const Faces<T> fa = faces_at(L, Cell{cgx, cgy, qr});
        const T d = L.kd ? L.kd[c] : fsum(fa);
        const T m = L.mm[c];
        const cx<T> diag = mk(fmaT(sft.re, m, d), mulT(sft.im, m));
        const cx<T> Az = diag * Zq[cr] - nb_sum3<T, RX>(L, fa, cgx, cgy, qr, cr, Zm, Zq, Zp, mk(T(0), T(0)));
        v = sF[(qr % R3F) * P + cr] - Az;
      }
      const int base = (tid & 31) & ~3;
      const cx<T> v0 = shfl_cx(v, base), v1 = shfl_cx(v, base + 1), v2 = shfl_cx(v, base + 2),
                  v3 = shfl_cx(v, base + 3);
      if (cvalid && (tid & 3) == 0) {
        cx<T> acc = (qr & 1) ? sC[ck] : mk(T(0), T(0));
        acc = acc + v0;
        acc = acc + v1;
        acc = acc + v2;
        acc = acc + v3;
        if (qr & 1) fcs[((int64_t)(qr >> 1) * cny + cY) * cnx + cX] = acc;
        else sC[ck] = acc;
      }
    }
    // phase 1d: ... and its first half sweep (red, from z = 0)
    if (load) {
      cx<T>* Fp = sF + (p % R3F) * P;
      cx<T>* Zp = sZ + (p % R3Z) * P;
#pragma unroll
      for (int u = 0; u < LOADS; ++u) {
        const int it = tid + u * NT;
        if (it < P) {
          Fp[it] = fv[u];
          if (red[u]) Zp[it] = iv[u] * fv[u];
        }
      }
    }
    if (p == plast) break;
    __syncthreads();
    sw_apply<T, TX, TY>(L, p - 1, s1, sZ, sF);
    __syncthreads();
    sw_apply<T, TX, TY>(L, p - 2, s2, sZ, sF);
    __syncthreads();
    sw_apply<T, TX, TY>(L, p - 3, s3, sZ, sF);
    __syncthreads();
  }
}

// post: phases at march step p
//   1: output of plane p - 5 (its red cells get the fourth half sweep here:
//      they read black of p - 6 .. p - 4, final) and load of plane p with the
//      interpolated coarse correction
//   2: black half sweep on p - 1 (reads red of p - 2 .. p: interpolated values;
//      red of p - 2 is updated only in phase 3)
//   3: red on p - 2 (reads black of p - 3 .. p - 1: first-sweep values)
//   4: black on p - 3 (reads red of p - 4 .. p - 2: second-sweep values; red of
//      p - 4 gets its last sweep only in phase 1 of step p + 1)
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(Tile3<TX, TY>::NT) k_post3d(LevelView<T> L, uint32_t mask, const SlotState* st,
                                                              const cx<T>* __restrict__ invd,
                                                              const cx<T>* __restrict__ f,
                                                              const cx<T>* __restrict__ z, cx<T>* __restrict__ zout,
                                                              int64_t vs, const cx<T>* __restrict__ zc, int64_t vsc,
                                                              z64* __restrict__ Zk, int64_t vsZk, int64_t zcol,
                                                              int zch) {
  constexpr int RX = Tile3<TX, TY>::RX, P = Tile3<TX, TY>::P, NT = Tile3<TX, TY>::NT;
  constexpr int LOADS = Tile3<TX, TY>::LOADS;
  extern __shared__ __align__(16) unsigned char post3_smem[];
  cx<T>* sZ = (cx<T>*)post3_smem;
  cx<T>* sF = sZ + R3Z * P;
  const int slot = blockIdx.z;
  if (!slot_running3(st, slot)) return;
  const int tau = st[slot].tau;
  const cx<T>* ID = invd + (int64_t)tau * L.n;
  const cx<T>* fs = f + slot * vs;
  const cx<T>* zs = z + slot * vs;
  cx<T>* zo = zout ? zout + slot * vs : nullptr;
  const cx<T>* zcs = zc + slot * vsc;
  z64* zk = Zk ? Zk + slot * vsZk + (int64_t)(st[slot].k - 1) * zcol : nullptr;
  const bool first = st[slot].cycles == 0;
  const int ntx = (L.nx + TX - 1) / TX;
  const int bx = blockIdx.x % ntx, by = blockIdx.x / ntx;
  const int x0 = bx * TX - FH, y0 = by * TY - FH;
  const int z0 = blockIdx.y * zch, z1 = min(z0 + zch, L.nz);
  const int cnx = L.nx >> 1, cny = L.ny >> 1, cnz = L.nz >> 1;
  const int tid = threadIdx.x;
  const int ox = tid % TX, oy = tid / TX;
  const int ogx = x0 + FH + ox, ogy = y0 + FH + oy;
  const bool own = tid < TX * TY && ogx < L.nx && ogy < L.ny;
  const int orr = (oy + FH) * RX + ox + FH;
  const int pfirst = max(z0 - FH, 0), plast = z1 + FH;
  for (int p = pfirst; p <= plast; ++p) {
    SwCell<T> s1, s2, s3;
    sw_fetch<T, TX, TY>(L, ID, x0, y0, p - 1, 1, 1, plane_in(p - 1, z0 - 3, z1 + 3, L.nz), s1);
    sw_fetch<T, TX, TY>(L, ID, x0, y0, p - 2, 0, 2, plane_in(p - 2, z0 - 2, z1 + 2, L.nz), s2);
    sw_fetch<T, TX, TY>(L, ID, x0, y0, p - 3, 1, 3, plane_in(p - 3, z0 - 1, z1 + 1, L.nz), s3);
    // phase 1a: load plane p (all loads first): f, and z + P z_coarse
    const bool load = plane_in(p, z0 - FH, z1 + FH, L.nz);
    cx<T> fv[LOADS], zv[LOADS];
#pragma unroll
    for (int u = 0; u < LOADS; ++u) {
      const int it = tid + u * NT;
      const int ry = it / RX, rx = it - ry * RX;
      const int gx = x0 + rx, gy = y0 + ry;
      const bool in = load && it < P && gx >= 0 && gx < L.nx && gy >= 0 && gy < L.ny;
      const int64_t c = ((int64_t)p * L.ny + gy) * L.nx + gx;
      fv[u] = mk(T(0), T(0));
      zv[u] = mk(T(0), T(0));
      if (in) {
        fv[u] = fs[c];
        zv[u] = zs[c] + prolong_value(Cell{gx, gy, p}, 2, 2, 2, cnx, cny, cnz, mask, zcs);
      }
    }
    // phase 1b: output of plane q = p - 5; red cells take the fourth half sweep
    const int qo = p - 5;
    if (qo >= z0 && qo < z1 && own) {
      const cx<T>* Zq = sZ + (qo % R3Z) * P;
      const int64_t c = ((int64_t)qo * L.ny + ogy) * L.nx + ogx;
      cx<T> v;
      if (((ogx + ogy + qo) & 1) == 0) {
        const cx<T>* Zm = sZ + ((qo + R3Z - 1) % R3Z) * P;
        const cx<T>* Zp = sZ + ((qo + 1) % R3Z) * P;
        const cx<T> rhs = nb_sum3<T, RX>(L, faces_at(L, Cell{ogx, ogy, qo}), ogx, ogy, qo, orr, Zm, Zq, Zp,
                                         sF[(qo % R3F) * P + orr]);
        v = ID[c] * rhs;
      } else {
        v = Zq[orr];
      }
      if (zk) {
        const z64 ev = cvt<double>(v);
        zk[c] = first ? ev : (zk[c] + ev);
      } else {
        zo[c] = v;
      }
    }
    if (load) {
      cx<T>* Fp = sF + (p % R3F) * P;
      cx<T>* Zp = sZ + (p % R3Z) * P;
#pragma unroll
      for (int u = 0; u < LOADS; ++u) {
        const int it = tid + u * NT;
        if (it < P) {
          Fp[it] = fv[u];
          Zp[it] = zv[u];
        }
      }
    }
    if (p == plast) break;
    __syncthreads();
    sw_apply<T, TX, TY>(L, p - 1, s1, sZ, sF);
    __syncthreads();
    sw_apply<T, TX, TY>(L, p - 2, s2, sZ, sF);
    __syncthreads();
    sw_apply<T, TX, TY>(L, p - 3, s3, sZ, sF);
    __syncthreads();
  }
}

// --------------------------------------------------------------------- launchers
template <typename T, int TX, int TY>
static size_t fused3_smem(bool pre) {
  return (size_t)(R3Z + R3F) * Tile3<TX, TY>::P * sizeof(cx<T>) + (pre ? (size_t)(TX / 2) * (TY / 2) * sizeof(cx<T>) : 0);
}

bool fused3d_level_ok(const LevelHost& L) {
  return L.nz > 1 && L.rx == 2 && L.ry == 2 && L.rz == 2 && L.nx % 2 == 0 && L.ny % 2 == 0 && L.nz % 2 == 0;
}

template <typename T>
void fused3d_prepare() {
  cudaFuncSetAttribute(k_pre3d<T, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fused3_smem<T, 8, 8>(true));
  cudaFuncSetAttribute(k_post3d<T, 8, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused3_smem<T, 8, 8>(false));
  cudaFuncSetAttribute(k_pre3d<T, 16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused3_smem<T, 16, 16>(true));
  cudaFuncSetAttribute(k_post3d<T, 16, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused3_smem<T, 16, 16>(false));
  cudaFuncSetAttribute(k_pre3d<T, 32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused3_smem<T, 32, 16>(true));
  cudaFuncSetAttribute(k_post3d<T, 32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)fused3_smem<T, 32, 16>(false));
}

static inline unsigned cdiv(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

template <typename T, int TX, int TY>
static void pre3_go(const LevelHost& F, const SlotState* st, const cx<T>* invd, const z64* taus, const cx<T>* f,
                    cx<T>* z, int64_t vs, cx<T>* fc, int64_t vsc, int nslot, int zc, cudaStream_t s) {
  dim3 g(cdiv(F.nx, TX) * cdiv(F.ny, TY), cdiv(F.nz, zc), nslot);
  k_pre3d<T, TX, TY><<<g, Tile3<TX, TY>::NT, fused3_smem<T, TX, TY>(true), s>>>(view<T>(F), st, invd, taus, f, z, vs, fc, vsc, zc);
}

template <typename T, int TX, int TY>
static void post3_go(const LevelHost& F, uint32_t mask, const SlotState* st, const cx<T>* invd, const cx<T>* f,
                     const cx<T>* z, cx<T>* zout, int64_t vs, const cx<T>* zc, int64_t vsc, int nslot, int zch,
                     cudaStream_t s, z64* Zk, int64_t vsZk, int64_t zcol) {
  dim3 g(cdiv(F.nx, TX) * cdiv(F.ny, TY), cdiv(F.nz, zch), nslot);
  k_post3d<T, TX, TY><<<g, Tile3<TX, TY>::NT, fused3_smem<T, TX, TY>(false), s>>>(view<T>(F), mask, st, invd, f, z, zout, vs, zc,
                                                                     vsc, Zk, vsZk, zcol, zch);
}

// z-chunk: an even number of planes (at least 2)
static int even_chunk(int zc, int nz) {
  zc = zc <= 0 ? nz : zc;
  zc = std::max(2, zc & ~1);
  return std::min(zc, nz);
}

template <typename T>
void launch_pre3d(const LevelHost& F, const SlotState* st, const cx<T>* invd, const z64* taus, const cx<T>* f,
                  cx<T>* z, int64_t vs, cx<T>* fc, int64_t vsc, int nslot, int tile, int zc, cudaStream_t s) {
  zc = even_chunk(zc, F.nz);
  if (tile == 8) pre3_go<T, 8, 8>(F, st, invd, taus, f, z, vs, fc, vsc, nslot, zc, s);
  else if (tile == 16) pre3_go<T, 16, 16>(F, st, invd, taus, f, z, vs, fc, vsc, nslot, zc, s);
  else pre3_go<T, 32, 16>(F, st, invd, taus, f, z, vs, fc, vsc, nslot, zc, s);
}

template <typename T>
void launch_post3d(const LevelHost& F, uint32_t mask, const SlotState* st, const cx<T>* invd, const cx<T>* f,
                   const cx<T>* z, cx<T>* zout, int64_t vs, const cx<T>* zc, int64_t vsc, int nslot, int tile,
                   int zch, cudaStream_t s, z64* Zk, int64_t vsZk, int64_t zcol) {
  zch = even_chunk(zch, F.nz);
  if (tile == 8) post3_go<T, 8, 8>(F, mask, st, invd, f, z, zout, vs, zc, vsc, nslot, zch, s, Zk, vsZk, zcol);
  else if (tile == 16) post3_go<T, 16, 16>(F, mask, st, invd, f, z, zout, vs, zc, vsc, nslot, zch, s, Zk, vsZk, zcol);
  else post3_go<T, 32, 16>(F, mask, st, invd, f, z, zout, vs, zc, vsc, nslot, zch, s, Zk, vsZk, zcol);
}

#define INST3(T)                                                                                                   \
  template void fused3d_prepare<T>();                                                                               \
  template void launch_pre3d<T>(const LevelHost&, const SlotState*, const cx<T>*, const z64*, const cx<T>*, cx<T>*, \
                                int64_t, cx<T>*, int64_t, int, int, int, cudaStream_t);                             \
  template void launch_post3d<T>(const LevelHost&, uint32_t, const SlotState*, const cx<T>*, const cx<T>*,          \
                                 const cx<T>*, cx<T>*, int64_t, const cx<T>*, int64_t, int, int, int, cudaStream_t, \
                                 z64*, int64_t, int64_t);
INST3(float)
INST3(double)

}  // namespace fks
