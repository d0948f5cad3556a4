// Device code for the two-component Shan-Chen D3Q19 evaporation step
// (arXiv:1701.03637, Sec. II) shared by all launches of the library.
//
// State between launches ("pre-stream" form): the buffer holds post-collision
// populations f*(t-1). One launch pulls them (streaming with halfway
// bounce-back), applies the evaporation sink to the arrived populations, forms
// densities and Psi, the Eq. (3) force, and collides (Eqs. (1), (2) with the
// tau F / rho velocity shift), writing f*(t) to the other buffer. The canonical
// (post-stream, post-sink) populations of step t are pull + sink of the buffer.
//
// Memory layout: 2 x 19 arrays (component-major, then direction) of np elements;
// site s = x + nx (y + ny z) with x fastest, rows contiguous without padding so
// that neighbouring tiles share every fetched sector through L2. Periodic wrap
// is index arithmetic.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

namespace sclbm {

constexpr int Q = 19;
constexpr int FLUID = 0, SINK = 1, SOLID = 2;

// D3Q19, own order: rest, +-x, +-y, +-z, then the 12 face diagonals in
// opposite pairs (i odd, i+1) with e_{i+1} = -e_i.
__host__ __device__ constexpr int dir_x(int i) {
  return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
       : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int dir_y(int i) {
  return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
       : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int dir_z(int i) {
  return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
       : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// e_y + 1 and e_z + 1 of all 19 directions in 2 bits each, for runtime direction indices.
constexpr unsigned long long pack_dir(int axis) {
  unsigned long long v = 0;
  for (int i = 0; i < 19; ++i)
    v |= (unsigned long long)((axis == 1 ? dir_y(i) : dir_z(i)) + 1) << (2 * i);
  return v;
}
constexpr unsigned long long kDirY = pack_dir(1), kDirZ = pack_dir(2);
__device__ __forceinline__ int dir_y_rt(int i) { return (int)((kDirY >> (2 * i)) & 3ull) - 1; }
__device__ __forceinline__ int dir_z_rt(int i) { return (int)((kDirZ >> (2 * i)) & 3ull) - 1; }
// Lattice weights (Sec. II A): 1/3 rest, 1/18 axis, 1/36 diagonal. In FP32 they are
// chosen within two ulps of those values so that w0 + 6 w1 + 12 w2 == 1 exactly:
// with the nearest floats the sum is 1 + 2^-26 and every collision would create
// that fraction of its mass (a steady drift of the conserved totals).
constexpr float kW1 = 14913080.0f * 0x1p-28f;  // 1/18 - 1 ulp
constexpr float kW2 = 7456540.0f * 0x1p-28f;   // kW1 / 2 exactly
constexpr float kW0 = 11184812.0f * 0x1p-25f;  // 1 - 12 kW1 exactly
__host__ __device__ constexpr float wgt(int i) { return i == 0 ? kW0 : (i <= 6 ? kW1 : kW2); }
__host__ __device__ constexpr double wgt_d(int i) { return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0); }

// Everything a launch needs to know about one lattice.
struct LatDev {
  int nx, ny, nz, nxny;
  long long np;            // elements between consecutive (component, direction) arrays
  float omega[2], tau[2];  // 1/tau and tau per component
  float G, rhoH;           // g of Eq. (3); imposed rho^r at sinks
  float Gs[2];             // self couplings g^{rr}, g^{bb} of Eq. (3) (0: the paper's two-component model)
  double rhoH_mass;        // exact sum of the reset r populations fl(w_i rho_H)
  int geometry, sink_z0, sink_layers;  // sink_z0 in [0, nz)
  double scx, scy, scz, RH2;
  int wall_z0, wall_z1;    // solid slab [wall_z0, wall_z1)
  // z-slab of a larger lattice: local plane z is plane (z + zoff) mod nzg of the lattice
  // whose geometry (sinks, walls, sphere) these fields describe; planes [own0, own1) are
  // the slab's own, the rest ghosts whose evaporation is not booked. A whole lattice has
  // zoff = 0, nzg = nz, own0 = 0, own1 = nz.
  int zoff, nzg, own0, own1;
};

// Plane of the whole lattice that local plane z is (z in [0, nz)).
__device__ __forceinline__ int global_z(const LatDev& L, int z) {
  int g = z + L.zoff;
  g = g >= L.nzg ? g - L.nzg : g;
  return g >= L.nzg ? g - L.nzg : g;
}
__device__ __forceinline__ bool own_z(const LatDev& L, int z) { return z >= L.own0 && z < L.own1; }

// ------------------------------------------------------------------ storage types
// ld: a population from global memory. pull_async: start a 4-byte asynchronous
// copy (cp.async, cached in L1) of the word holding a population into shared
// memory and return which half of the word it is (16-bit types). word: the
// population from such a word.
__device__ __forceinline__ void cp_async4(uint32_t* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
// 16-byte asynchronous copy kept in L2 only (each row is read once per CTA).
// Both addresses must be 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// ldcg: a population read at L2 only (ld.global.cg), never from L1, for kernels in
// which other CTAs of the same launch overwrite the data between two reads.
struct StF32 {
  using T = float;
  static __device__ __forceinline__ float ld(const T* p, float) { return __ldg(p); }
  static __device__ __forceinline__ float ldcg(const T* p, float) { return __ldcg(p); }
  static __device__ __forceinline__ float cv(T v, float) { return v; }
  static __device__ __forceinline__ void st(T* p, float v, float) { *p = v; }
  static __device__ __forceinline__ uint32_t pull_async(uint32_t* sm, const T* p) {
    cp_async4(sm, p);
    return 0u;
  }
  static __device__ __forceinline__ float word(uint32_t w, uint32_t, float) { return __uint_as_float(w); }
};
// FP16 / BF16 offsets h = f - w_i * rho0 (rho0 = 1), round to nearest even.
// Arrays hold an even number of elements, so the aligned word of any element
// lies inside its array.
template <class Half>
__device__ __forceinline__ uint32_t pull_async16(uint32_t* sm, const Half* p) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p);
  cp_async4(sm, reinterpret_cast<const void*>(a & ~uintptr_t(3)));
  return (uint32_t)(a >> 1) & 1u;
}
__device__ __forceinline__ unsigned short ldcg16(const void* p) {
  return __ldcg(reinterpret_cast<const unsigned short*>(p));
}
struct StF16 {
  using T = __half;
  static __device__ __forceinline__ float ld(const T* p, float w) { return w + __half2float(__ldg(p)); }
  static __device__ __forceinline__ float ldcg(const T* p, float w) { return w + __half2float(__ushort_as_half(ldcg16(p))); }
  static __device__ __forceinline__ float cv(T v, float w) { return w + __half2float(v); }
  static __device__ __forceinline__ void st(T* p, float v, float w) { *p = __float2half_rn(v - w); }
  static __device__ __forceinline__ uint32_t pull_async(uint32_t* sm, const T* p) { return pull_async16(sm, p); }
  static __device__ __forceinline__ float word(uint32_t w, uint32_t hi, float wt) {
    return wt + __half2float(__ushort_as_half((unsigned short)(hi ? w >> 16 : w & 0xffffu)));
  }
};
// FP16 of the population scaled by its weight, g = f_i / w_i (about rho),
// round to nearest even: the same relative spacing in the liquid and the vapour.
struct StF16S {
  using T = __half;
  static __device__ __forceinline__ float ld(const T* p, float w) { return __fmul_rn(w, __half2float(__ldg(p))); }
  static __device__ __forceinline__ float ldcg(const T* p, float w) {
    return __fmul_rn(w, __half2float(__ushort_as_half(ldcg16(p))));
  }
  static __device__ __forceinline__ float cv(T v, float w) { return __fmul_rn(w, __half2float(v)); }
  // w is a compile-time weight at every call, so 1 / w folds to a constant
  static __device__ __forceinline__ void st(T* p, float v, float w) { *p = __float2half_rn(__fmul_rn(v, 1.0f / w)); }
  static __device__ __forceinline__ uint32_t pull_async(uint32_t* sm, const T* p) { return pull_async16(sm, p); }
  static __device__ __forceinline__ float word(uint32_t w, uint32_t hi, float wt) {
    return __fmul_rn(wt, __half2float(__ushort_as_half((unsigned short)(hi ? w >> 16 : w & 0xffffu))));
  }
};
struct StBF16 {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float ld(const T* p, float w) { return w + __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ float ldcg(const T* p, float w) {
    return w + __bfloat162float(__ushort_as_bfloat16(ldcg16(p)));
  }
  static __device__ __forceinline__ float cv(T v, float w) { return w + __bfloat162float(v); }
  static __device__ __forceinline__ void st(T* p, float v, float w) { *p = __float2bfloat16_rn(v - w); }
  static __device__ __forceinline__ uint32_t pull_async(uint32_t* sm, const T* p) { return pull_async16(sm, p); }
  static __device__ __forceinline__ float word(uint32_t w, uint32_t hi, float wt) {
    return wt + __bfloat162float(__ushort_as_bfloat16((unsigned short)(hi ? w >> 16 : w & 0xffffu)));
  }
};

__host__ __device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}
// Periodic wrap without a division when v is within one period of [0, n).
__host__ __device__ __forceinline__ int wrap_near(int v, int n) {
  v = v < 0 ? v + n : (v >= n ? v - n : v);
  return (unsigned)v < (unsigned)n ? v : wrapi(v, n);
}

__device__ __forceinline__ bool solid_z(const LatDev& L, int z) {
  const int g = global_z(L, z);
  return g >= L.wall_z0 && g < L.wall_z1;
}

// Site class from coordinates (no storage): solid slab, planar or spherical sink.
// The squared distance is formed without FMA contraction so it rounds like a
// plain host evaluation. z is a local plane; the geometry is the whole lattice's.
__device__ __forceinline__ int site_class(const LatDev& L, int x, int y, int zl) {
  if (solid_z(L, zl)) return SOLID;
  const int z = global_z(L, zl);
  if (L.geometry == 1) {
    const int dz = z - L.sink_z0;  // sink_z0 in [0, nzg), z in [0, nzg)
    return (dz < 0 ? dz + L.nzg : dz) < L.sink_layers ? SINK : FLUID;
  }
  if (L.geometry == 2) {
    const double dx = (double)x - L.scx, dy = (double)y - L.scy, dz = (double)z - L.scz;
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 >= L.RH2 ? SINK : FLUID;
  }
  return FLUID;
}

template <int I, int N>
struct Unroll {
  template <class F>
  static __device__ __forceinline__ void run(F&& f) {
    f(std::integral_constant<int, I>());
    Unroll<I + 1, N>::run(f);
  }
};
template <int N>
struct Unroll<N, N> {
  template <class F>
  static __device__ __forceinline__ void run(F&&) {}
};

// Source offsets of the pull for site (x, y, z): the population arriving in
// direction i comes from x - e_i (periodic); from a solid site it is the site's
// own opposite population (halfway bounce-back).
struct PullIdx {
  int xs[3], ys[3], zs[3];  // indexed by 1 + e (source = x - e)
  bool sol_m, sol_p;        // source plane z - 1 / z + 1 is solid
  int s;
  __device__ __forceinline__ PullIdx(const LatDev& L, int x, int y, int z) {
    const int xm = x == 0 ? L.nx - 1 : x - 1, xp = x == L.nx - 1 ? 0 : x + 1;
    const int ym = y == 0 ? L.ny - 1 : y - 1, yp = y == L.ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? L.nz - 1 : z - 1, zp = z == L.nz - 1 ? 0 : z + 1;
    xs[0] = xp; xs[1] = x; xs[2] = xm;
    ys[0] = yp * L.nx; ys[1] = y * L.nx; ys[2] = ym * L.nx;
    zs[0] = zp * L.nxny; zs[1] = z * L.nxny; zs[2] = zm * L.nxny;
    sol_p = solid_z(L, zp);
    sol_m = solid_z(L, zm);
    s = x + ys[1] + zs[1];
  }
  template <int I>
  __device__ __forceinline__ void at(int& idx, int& d) const {
    constexpr int ex = dir_x(I), ey = dir_y(I), ez = dir_z(I);
    const bool sol = ez > 0 ? sol_m : (ez < 0 ? sol_p : false);
    idx = sol ? s : xs[1 + ex] + ys[1 + ey] + zs[1 + ez];
    d = sol ? opp(I) : I;
  }
};

template <class S>
__device__ __forceinline__ void pull_full(const LatDev& L, const typename S::T* __restrict__ src, const PullIdx& P,
                                          float (&fr)[Q], float (&fb)[Q]) {
  const long long cstride = (long long)Q * L.np;
  Unroll<0, Q>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int idx, d;
    P.template at<I>(idx, d);
    const typename S::T* p = src + (long long)d * L.np + idx;
    fr[I] = S::ld(p, wgt(I));
    fb[I] = S::ld(p + cstride, wgt(I));
  });
}

// Asynchronous form of pull_full: population (c, i) goes to sm[(c Q + i) stride];
// bit i of the result says which half of the word holds direction i.
template <class S>
__device__ __forceinline__ uint32_t pull_async(const LatDev& L, const typename S::T* __restrict__ src,
                                               const PullIdx& P, uint32_t* sm, int stride) {
  const long long cstride = (long long)Q * L.np;
  uint32_t hi = 0u;
  Unroll<0, Q>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int idx, d;
    P.template at<I>(idx, d);
    const typename S::T* p = src + (long long)d * L.np + idx;
    hi |= S::pull_async(sm + I * stride, p) << I;
    S::pull_async(sm + (Q + I) * stride, p + cstride);
  });
  return hi;
}

// Density from the 19 populations of a site: opposite pairs (I, I+1) first, then
// a balanced tree (depth 5, so the additions overlap), in one fixed order that
// every kernel uses; get(i) yields population i, so values can be summed as they
// are loaded.
template <class Get>
__device__ __forceinline__ float sum19_of(Get&& get) {
  auto pair = [&](auto ic) {
    constexpr int I = 1 + 2 * decltype(ic)::value;
    return __fadd_rn(get(std::integral_constant<int, I>()), get(std::integral_constant<int, I + 1>()));
  };
  using std::integral_constant;
  const float c0 = __fadd_rn(pair(integral_constant<int, 0>()), pair(integral_constant<int, 1>()));
  const float c1 = __fadd_rn(pair(integral_constant<int, 2>()), pair(integral_constant<int, 3>()));
  const float c2 = __fadd_rn(pair(integral_constant<int, 4>()), pair(integral_constant<int, 5>()));
  const float c3 = __fadd_rn(pair(integral_constant<int, 6>()), pair(integral_constant<int, 7>()));
  const float c4 = __fadd_rn(pair(integral_constant<int, 8>()), get(integral_constant<int, 0>()));
  return __fadd_rn(__fadd_rn(__fadd_rn(c0, c1), __fadd_rn(c2, c3)), c4);
}
__device__ __forceinline__ float sum19(const float (&f)[Q]) {
  return sum19_of([&](auto ic) { return f[decltype(ic)::value]; });
}

// Evaporation boundary (Sec. II C) on the densities of the arrived populations:
// rho^r := rho_H, rho^b := rho^r + rho^b - rho_H.
__device__ __forceinline__ void sink_densities(const LatDev& L, float& rr, float& rb) {
  const float rbn = (rr + rb) - L.rhoH;
  rr = L.rhoH;
  rb = rbn;
}

// Reset value of direction i for density rho (f^eq at rest), an exact float product.
__device__ __forceinline__ float rest_pop(int i, float rho) { return __fmul_rn(wgt(i), rho); }

// Evaporated mass of one sink site: sum_i (f_i^r - w_i rho_H) over the arrived r
// populations, without contraction, so that where only reset values arrived (inside
// the sink region) every term is exactly zero and no rounding bias is booked.
__device__ __forceinline__ float sink_excess(const LatDev& L, const float (&fr)[Q]) {
  float e = 0.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) e = __fadd_rn(e, __fsub_rn(fr[i], rest_pop(i, L.rhoH)));
  return e;
}

// Eq. (4) with rho0 = 1. Below rho = 2^-6, 1 - exp(-rho) would cancel, so Psi
// is its Taylor series rho (1 - rho/2 (1 - rho/3 (1 - rho/4))) there (relative
// truncation below rho^4 / 120 <= 5e-10): trace densities keep Psi ~ rho.
__device__ __forceinline__ float psi_of(float rho) {
  if (rho < 0.015625f) {
    const float t = __fmaf_rn(-0.25f * rho, 1.0f / 3.0f, 1.0f / 3.0f);  // (1 - rho/4) / 3
    const float u = __fmaf_rn(-rho * 0.5f, t, 0.5f);                     // (1 - rho/3 (...)) / 2
    return __fmul_rn(rho, __fmaf_rn(-rho, u, 1.0f));
  }
  return 1.0f - expf(-rho);
}

template <class S>
__device__ __forceinline__ void store_site(const LatDev& L, typename S::T* __restrict__ dst, int s,
                                           const float (&fr)[Q], const float (&fb)[Q]) {
  const long long cstride = (long long)Q * L.np;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    typename S::T* p = dst + (long long)i * L.np + s;
    S::st(p, fr[i], wgt(i));
    S::st(p + cstride, fb[i], wgt(i));
  }
}

// Momentum sum_i f_i e_i of one component.
// Momentum sum_i f_i e_i of one component from the differences of opposite
// pairs, d = f_I - f_{I+1} (e_{I+1} = -e_I): each axis sums the five d whose
// e_I has a component along it.
__device__ __forceinline__ void momentum(const float (&f)[Q], float (&m)[3]) {
  float d[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) d[k] = __fsub_rn(f[1 + 2 * k], f[2 + 2 * k]);
  bool first[3] = {true, true, true};
  Unroll<0, 9>::run([&](auto kc) {
    constexpr int K = decltype(kc)::value, I = 1 + 2 * K;
    constexpr int e[3] = {dir_x(I), dir_y(I), dir_z(I)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (e[a] == 0) continue;
      if (first[a]) m[a] = e[a] > 0 ? d[K] : -d[K];
      else m[a] = e[a] > 0 ? __fadd_rn(m[a], d[K]) : __fsub_rn(m[a], d[K]);
      first[a] = false;
    }
  });
}

// The collision arithmetic below spells out every rounding (__fmul_rn, __fmaf_rn,
// ...) so that the compiler cannot contract it differently in different kernels:
// every step kernel produces the same bits for the same state.

// Common velocity u' = sum_c (m^c / tau_c) / sum_c (rho^c / tau_c) (Sec. II A: the
// mass-weighted u_eq when tau_r = tau_b).
__device__ __forceinline__ void common_velocity(const LatDev& L, float rr, float rb, const float (&mr)[3],
                                                const float (&mb)[3], float (&up)[3]) {
  const float omr = L.omega[0], omb = L.omega[1];
  const float den = __fmaf_rn(rr, omr, __fmul_rn(rb, omb));
  const float inv = den > 0.0f ? __fdiv_rn(1.0f, den) : 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) up[d] = __fmul_rn(__fmaf_rn(mr[d], omr, __fmul_rn(mb[d], omb)), inv);
}

// c . u for a D3Q19 direction, summing the non-zero terms in x, y, z order.
template <int I>
__device__ __forceinline__ float cdot(const float (&u)[3]) {
  constexpr int ex = dir_x(I), ey = dir_y(I), ez = dir_z(I);
  float r = 0.0f;
  bool first = true;
  if (ex != 0) { r = ex > 0 ? u[0] : -u[0]; first = false; }
  if (ey != 0) { r = first ? (ey > 0 ? u[1] : -u[1]) : (ey > 0 ? __fadd_rn(r, u[1]) : __fsub_rn(r, u[1])); first = false; }
  if (ez != 0) { r = first ? (ez > 0 ? u[2] : -u[2]) : (ez > 0 ? __fadd_rn(r, u[2]) : __fsub_rn(r, u[2])); }
  return r;
}

// Shifted-velocity BGK relaxation of component c at a fluid site (Eqs. (1)-(3)):
// u_eq = u' + tau_c F^c / rho^c with F^c = -Psi^c(x) g A: g = G and A = a^cbar =
// sum_i w_i Psi^cbar(x + e_i) e_i in the paper's two-component model, g = 1 and
// A = sum_cbar g^{c cbar} a^cbar (coupled_sums) with self couplings.
__device__ __forceinline__ void relax_core(float om, float tau, float (&f)[Q], float rho, float ps, float g,
                                           const float (&A)[3], const float (&up)[3]) {
  // tau F / rho = (-g tau) (Psi / rho) A with Psi / rho <= 1, so a trace (or
  // denormal) density cannot overflow the shift; rho = 0 takes u' itself
  const float q = rho > 0.0f ? __fdiv_rn(ps, rho) : 0.0f;
  const float gq = __fmul_rn(__fmul_rn(-g, tau), q);
  float u[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) u[d] = __fmaf_rn(gq, A[d], up[d]);
  const float usq = __fmaf_rn(u[0], u[0], __fmaf_rn(u[1], u[1], __fmul_rn(u[2], u[2])));
  const float base = __fmaf_rn(-1.5f, usq, 1.0f);  // 1 - 1.5 u.u
  // f^eq_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u); opposite directions share
  // the even part w rho (1 - 1.5 u.u) + 4.5 w rho (c.u)^2 and differ in the sign of
  // the odd part 3 w rho c.u. The factors of w rho are formed once per weight class.
  f[0] = __fmaf_rn(om, __fsub_rn(__fmul_rn(__fmul_rn(kW0, rho), base), f[0]), f[0]);
  const float wr1 = __fmul_rn(kW1, rho), wr2 = __fmul_rn(kW2, rho);
  const float wb1 = __fmul_rn(wr1, base), wb2 = __fmul_rn(wr2, base);
  const float w451 = __fmul_rn(4.5f, wr1), w452 = __fmul_rn(4.5f, wr2);
  const float w31 = __fmul_rn(3.0f, wr1), w32 = __fmul_rn(3.0f, wr2);
  Unroll<0, 9>::run([&](auto kc) {
    constexpr int I = 1 + 2 * decltype(kc)::value, J = I + 1;
    constexpr bool axis = I <= 6;
    const float cu = cdot<I>(u);
    const float ev = __fmaf_rn(__fmul_rn(axis ? w451 : w452, cu), cu, axis ? wb1 : wb2);
    const float od = __fmul_rn(axis ? w31 : w32, cu);
    f[I] = __fmaf_rn(om, __fsub_rn(__fadd_rn(ev, od), f[I]), f[I]);
    f[J] = __fmaf_rn(om, __fsub_rn(__fsub_rn(ev, od), f[J]), f[J]);
  });
}
__device__ __forceinline__ void relax(const LatDev& L, int c, float (&f)[Q], float rho, float ps, float g,
                                      const float (&A)[3], const float (&up)[3]) {
  relax_core(c == 0 ? L.omega[0] : L.omega[1], c == 0 ? L.tau[0] : L.tau[1], f, rho, ps, g, A, up);
}

// A^c = sum_cbar g^{c cbar} a^cbar of Eq. (3): the cross coupling g (= g^{rb} = g^{br})
// times the other component's sum, plus the self coupling g^{cc} times its own
// (an exact zero when g^{cc} = 0, the paper's two-component model).
__device__ __forceinline__ void coupled_sums(const LatDev& L, const float (&ar)[3], const float (&ab)[3],
                                             float (&Ar)[3], float (&Ab)[3]) {
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    Ar[d] = __fmaf_rn(L.Gs[0], ar[d], __fmul_rn(L.G, ab[d]));
    Ab[d] = __fmaf_rn(L.Gs[1], ab[d], __fmul_rn(L.G, ar[d]));
  }
}

// Shifted-velocity BGK collision of one fluid site, in place on fr/fb.
// ar/ab: sum_i w_i Psi^{r|b}(x + e_i) e_i.
__device__ __forceinline__ void collide(const LatDev& L, float (&fr)[Q], float (&fb)[Q], float rr, float rb, float psr,
                                        float psb, const float (&ar)[3], const float (&ab)[3]) {
  float mr[3], mb[3], up[3];
  momentum(fr, mr);
  momentum(fb, mb);
  common_velocity(L, rr, rb, mr, mb, up);
  if (L.Gs[0] == 0.0f && L.Gs[1] == 0.0f) {  // the paper's model: the cross coupling alone
    relax(L, 0, fr, rr, psr, L.G, ab, up);
    relax(L, 1, fb, rb, psb, L.G, ar, up);
  } else {
    float Ar[3], Ab[3];
    coupled_sums(L, ar, ab, Ar, Ab);
    relax(L, 0, fr, rr, psr, 1.0f, Ar, up);
    relax(L, 1, fb, rb, psb, 1.0f, Ab, up);
  }
}

// sum_i w_i Psi^c(x + e_i) e_i of both components from a Psi ring whose cells hold
// (Psi^r, Psi^b); psi2(plane slot, ly, lx). Opposite pairs (I, I+1) contribute
// w_I (Psi(x + e_I) - Psi(x - e_I)) e_I.
template <class PsiAt2>
__device__ __forceinline__ void force_sums(PsiAt2 psi2, int sm1, int s0, int sp1, int ly, int lx, float (&ar)[3],
                                           float (&ab)[3]) {
  ar[0] = ar[1] = ar[2] = 0.f;
  ab[0] = ab[1] = ab[2] = 0.f;
  Unroll<0, 9>::run([&](auto kc) {
    constexpr int I = 1 + 2 * decltype(kc)::value;
    constexpr int ex = dir_x(I), ey = dir_y(I), ez = dir_z(I);
    const int sa = ez > 0 ? sp1 : (ez < 0 ? sm1 : s0);
    const int sb = ez > 0 ? sm1 : (ez < 0 ? sp1 : s0);
    const float2 pa = psi2(sa, ly + ey, lx + ex), pb = psi2(sb, ly - ey, lx - ex);
    const float dr = __fsub_rn(pa.x, pb.x), db = __fsub_rn(pa.y, pb.y);
    auto acc = [&](float& a, int e, float d) { a = __fmaf_rn(e > 0 ? wgt(I) : -wgt(I), d, a); };
    if (ex != 0) { acc(ar[0], ex, dr); acc(ab[0], ex, db); }
    if (ey != 0) { acc(ar[1], ey, dr); acc(ab[1], ey, db); }
    if (ez != 0) { acc(ar[2], ez, dr); acc(ab[2], ez, db); }
  });
}

// sum_i w_i Psi(x + e_i) e_i of one component, with force_sums' order of operations;
// psi1(plane slot, ly, lx) yields that component's Psi.
template <class PsiAt1>
__device__ __forceinline__ void force_sum_one(PsiAt1 psi1, int sm1, int s0, int sp1, int ly, int lx, float (&a)[3]) {
  a[0] = a[1] = a[2] = 0.f;
  Unroll<0, 9>::run([&](auto kc) {
    constexpr int I = 1 + 2 * decltype(kc)::value;
    constexpr int ex = dir_x(I), ey = dir_y(I), ez = dir_z(I);
    const int sa = ez > 0 ? sp1 : (ez < 0 ? sm1 : s0);
    const int sb = ez > 0 ? sm1 : (ez < 0 ? sp1 : s0);
    const float d = __fsub_rn(psi1(sa, ly + ey, lx + ex), psi1(sb, ly - ey, lx - ex));
    auto acc = [&](float& v, int e) { v = __fmaf_rn(e > 0 ? wgt(I) : -wgt(I), d, v); };
    if (ex != 0) acc(a[0], ex);
    if (ey != 0) acc(a[1], ey);
    if (ez != 0) acc(a[2], ez);
  });
}

// ------------------------------------------------------------------ fused step, one x-y tile column
//
// A CTA of TX*TY threads owns sites [x0, x0+TX) x [y0, y0+TY) and marches z over
// [zb, ze). Psi of the tile plus a one-site halo lives in a 4-plane shared ring,
// so the 18-neighbour force never reads Psi from HBM; halo densities are
// recomputed from the neighbours' pulled populations (an L2 hit when the
// neighbouring CTA is at the same plane). Halo slot h belongs to thread h: the
// two halo rows each fill a warp with contiguous sites, so their pulls coalesce
// like the interior's (spreading them over all warps instead made every halo
// load touch a sector per lane). One barrier per plane: plane z+1 is written
// while plane z-2's slot is free.
//
// The pulls of the next plane are asynchronous copies into shared slots that
// belong to the issuing thread alone (its site's 38 populations, and its halo
// site's), started as soon as the current plane has been read out of them, so
// their latency overlaps the collision of the previous plane without holding
// registers. Only the thread that issued a copy reads its slot, so a wait on its
// own copies is the only synchronisation the slots need.
template <int TX, int TY, class S>
struct Tile {
  static constexpr int NT = TX * TY, NW = NT / 32, RW = TX + 2, RH = TY + 2, NH = 2 * TX + 2 * RH;
  static constexpr int HS = (NH + 31) / 32 * 32;  // halo slot stride
  static_assert(NH <= NT, "halo slots exceed threads");
  static_assert(NT % 32 == 0, "whole warps");

  struct Smem {
    float2 ring[4][RH][RW];  // (Psi^r, Psi^b) of plane slot, tile row + 1, tile column + 1
    double red[NW];
    uint32_t fin[2 * Q][NT];       // pulled populations of the own site, [c Q + i][thread]
    uint32_t fh[2 * Q][HS];        // pulled populations of the halo site, [c Q + i][thread]
  };

  const LatDev& L;
  Smem& sm;
  const typename S::T* __restrict__ src;
  typename S::T* __restrict__ dst;
  int tx, ty, x, y, hx, hy, hlx, hly;
  bool active, has_halo;
  double evap;

  __device__ __forceinline__ Tile(const LatDev& L_, Smem& sm_, const typename S::T* s_, typename S::T* d_)
      : L(L_), sm(sm_), src(s_), dst(d_), evap(0.0) {}

  __device__ __forceinline__ int wrapz(int z) const { return z < 0 ? z + L.nz : (z >= L.nz ? z - L.nz : z); }
  __device__ __forceinline__ uint32_t* own_slot() { return &sm.fin[0][threadIdx.x]; }
  __device__ __forceinline__ uint32_t* halo_slot() { return &sm.fh[0][threadIdx.x]; }

  // Bind the CTA to tile column (bx, by). Lanes past a ragged edge stage the
  // wrapped site there (its Psi is the halo of the last real site).
  __device__ __forceinline__ void setup(int bx, int by) {
    const int tid = threadIdx.x;
    tx = tid % TX;
    ty = tid / TX;
    const int gx = bx * TX + tx, gy = by * TY + ty;
    active = gx < L.nx && gy < L.ny;
    x = gx % L.nx;
    y = gy % L.ny;
    // halo slot h = tid: top row, bottom row, left column, right column
    const int h = tid;
    has_halo = h < NH;
    if (h < TX) { hlx = h; hly = -1; }
    else if (h < 2 * TX) { hlx = h - TX; hly = TY; }
    else if (h < 2 * TX + RH) { hlx = -1; hly = h - 2 * TX - 1; }
    else { hlx = TX; hly = h - 2 * TX - RH - 1; }
    hx = wrapi(bx * TX + hlx, L.nx);
    hy = wrapi(by * TY + hly, L.ny);
  }

  // Start the pulls of plane p (p in [-1, nz]) for the own site and the halo site.
  __device__ __forceinline__ void issue(int p, int& cls, uint32_t& hi, int& hcl, uint32_t& hhi) {
    const int zp = wrapz(p);
    cls = site_class(L, x, y, zp);
    if (cls != SOLID) hi = pull_async<S>(L, src, PullIdx(L, x, y, zp), own_slot(), NT);
    if (has_halo) {
      hcl = site_class(L, hx, hy, zp);
      if (hcl != SOLID) hhi = pull_async<S>(L, src, PullIdx(L, hx, hy, zp), halo_slot(), HS);
    }
    cp_async_commit();
  }

  // Read plane p out of the slots (after the wait): the own site into fr/fb, the
  // halo site as sums; apply the sink and publish Psi to ring slot p & 3.
  __device__ __forceinline__ void take(int p, bool own, int cls, uint32_t hi, int hcl, uint32_t hhi,
                                       float (&fr)[Q], float (&fb)[Q], float& rr, float& rb) {
    const int slot = p & 3;
    float pr = 0.0f, pb = 0.0f;
    if (cls == SOLID) {
      rr = rb = 0.0f;
    } else {
      const uint32_t* w = own_slot();
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        const uint32_t h = (hi >> i) & 1u;
        fr[i] = S::word(w[i * NT], h, wgt(i));
        fb[i] = S::word(w[(Q + i) * NT], h, wgt(i));
      }
      rr = sum19(fr);
      rb = sum19(fb);
      if (cls == SINK) {
        if (active && own && own_z(L, wrapz(p))) evap += (double)sink_excess(L, fr);
        sink_densities(L, rr, rb);
      }
      pr = psi_of(rr);
      pb = psi_of(rb);
    }
    sm.ring[slot][ty + 1][tx + 1] = make_float2(pr, pb);
    if (has_halo) {
      float hpr = 0.0f, hpb = 0.0f;
      if (hcl != SOLID) {
        const uint32_t* w = halo_slot();
        // the owner's arithmetic, so the halo Psi has the owner's bits
        float hrr = sum19_of([&](auto ic) {
          constexpr int I = decltype(ic)::value;
          return S::word(w[I * HS], (hhi >> I) & 1u, wgt(I));
        });
        float hrb = sum19_of([&](auto ic) {
          constexpr int I = decltype(ic)::value;
          return S::word(w[(Q + I) * HS], (hhi >> I) & 1u, wgt(I));
        });
        if (hcl == SINK) sink_densities(L, hrr, hrb);
        hpr = psi_of(hrr);
        hpb = psi_of(hrb);
      }
      sm.ring[slot][hly + 1][hlx + 1] = make_float2(hpr, hpb);
    }
  }

  // Collide plane z (in [0, nz); read out one plane earlier) and store f*.
  __device__ __forceinline__ void finish(int z, float (&fr)[Q], float (&fb)[Q], float rr, float rb, int cls) {
    if (!active || cls == SOLID) return;
    const int s = x + L.nx * y + L.nxny * z;
    if (cls == SINK) {
      // Sinks are neither forced nor collided: they stream f^eq(rho_H, 0) and
      // f^eq(rho^r + rho^b - rho_H, 0) as they are.
#pragma unroll
      for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, rr); fb[i] = rest_pop(i, rb); }
    } else {
      float ar[3], ab[3];
      auto psi2 = [&](int sl, int ly, int lx) { return sm.ring[sl][ly + 1][lx + 1]; };
      force_sums(psi2, (z - 1) & 3, z & 3, (z + 1) & 3, ty, tx, ar, ab);
      const float2 ps = sm.ring[z & 3][ty + 1][tx + 1];
      collide(L, fr, fb, rr, rb, ps.x, ps.y, ar, ab);
    }
    store_site<S>(L, dst, s, fr, fb);
  }

  // March planes [zb, ze) upward (down = false) or downward. Plane p is read out
  // of the slots at step o, its successor's pulls are started, and after the
  // barrier plane p - d (whose Psi neighbours are now all in the ring) collides.
  // The halo plane on each end is staged for Psi only. The ring slot of plane
  // p is p & 3 for p = -1 too, as in finish().
  __device__ __forceinline__ void run(int zb, int ze, bool down) {
    float cr[Q], cb[Q], nr[Q], nb[Q];
    float crr = 0.f, crb = 0.f, nrr = 0.f, nrb = 0.f;
    int ccl = SOLID, ncl = SOLID, hcl = SOLID;
    uint32_t hi = 0u, hhi = 0u;
    const int d = down ? -1 : 1;
    const int first = down ? ze - 1 : zb;
    const int n = ze - zb;
    issue(first - d, ncl, hi, hcl, hhi);
    for (int o = 0; o < n + 2; ++o) {
      const int p = first + (o - 1) * d;
      cp_async_wait_all();
      take(p, o >= 1 && o <= n, ncl, hi, hcl, hhi, nr, nb, nrr, nrb);
      const int pcl = ncl;
      if (o + 1 < n + 2) issue(p + d, ncl, hi, hcl, hhi);
      __syncthreads();
      if (o >= 2) finish(p - d, cr, cb, crr, crb, ccl);
#pragma unroll
      for (int i = 0; i < Q; ++i) { cr[i] = nr[i]; cb[i] = nb[i]; }
      crr = nrr;
      crb = nrb;
      ccl = pcl;
    }
  }

  // Block sum of the evaporated mass (fixed order: warps, then warp 0's lanes).
  __device__ __forceinline__ double block_evap() {
    double v = evap;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
      for (int k = 0; k < NT / 32; ++k) t += sm.red[k];
    return t;
  }
};

// ------------------------------------------------------------------ fused step, staged rows
//
// The same march as Tile, with the pulls staged cooperatively. For each of the
// 38 (component, direction) pairs the plane's source rows -- the TY + 2 rows
// y0 - 1 .. y0 + TY shifted by -e_y, in plane z - e_z -- are copied into shared
// memory over columns x0 - E .. x0 + TX + E as aligned 16-byte chunks (E
// populations each), and the x shift -e_x is applied when a thread reads them.
// The E-column margins hold the side halo, so the halo needs no pulls of its
// own. Chunks are spread evenly over the CTA's threads (a per-plane table holds
// each row's offset, a per-column table each chunk's wrapped x), so no warp
// carries more copy work than another. Requires nx % E == 0 (then every
// wrapped chunk is aligned). A population whose source plane is solid is the
// site's own opposite population (halfway bounce-back): read directly.
//
// Per plane: wait for the copies, barrier, read out plane p (Psi to the ring,
// own populations to registers), write the row table of plane p + d, barrier,
// start plane p + d's copies, collide plane p - d.
template <int TX, int TY, class S>
struct TileRows {
  using T = typename S::T;
  static constexpr int E = 16 / (int)sizeof(T);           // populations per chunk
  static constexpr int NT = TX * TY, NW = NT / 32, RW = TX + 2, RH = TY + 2, NH = 2 * TX + 2 * RH;
  static constexpr int SW = TX + 2 * E;                   // staged row width
  static constexpr int CH = SW / E;                       // chunks per row
  static constexpr int NR = 2 * Q * RH;                   // staged rows per plane
  static constexpr int RS = NT / CH;                      // rows copied per pass of the CTA
  static_assert(TX % E == 0, "tile width must be a multiple of the chunk");
  static_assert(NH <= NT && NT % 32 == 0, "tile shape");

  struct Smem {
    T stage[2 * Q][RH][SW];  // rows of plane p: [c Q + i][y - y0 + 1][x - x0 + E]
    float2 ring[4][RH][RW];  // (Psi^r, Psi^b) of plane slot, tile row + 1, tile column + 1
    const T* rowp[NR];       // source address of each staged row's column x = 0
    int chx[CH];             // wrapped x of chunk j
    double red[NW];
  };

  const LatDev& L;
  Smem& sm;
  const T* __restrict__ src;
  T* __restrict__ dst;
  int tx, ty, x, y, hx, hy, hlx, hly, y0;
  int cr0, cj;  // this thread's copy work: rows cr0, cr0 + RS, ... at chunk cj (cr0 >= NR: none)
  bool active, has_halo;
  double evap;

  __device__ __forceinline__ TileRows(const LatDev& L_, Smem& sm_, const T* s_, T* d_)
      : L(L_), sm(sm_), src(s_), dst(d_), evap(0.0) {}

  __device__ __forceinline__ int wrapz(int z) const { return z < 0 ? z + L.nz : (z >= L.nz ? z - L.nz : z); }

  __device__ __forceinline__ void setup(int bx, int by) {
    const int tid = threadIdx.x;
    tx = tid % TX;
    ty = tid / TX;
    const int gx = bx * TX + tx, gy = by * TY + ty;
    active = gx < L.nx && gy < L.ny;
    x = gx % L.nx;
    y = gy % L.ny;
    y0 = by * TY;
    const int h = tid;  // halo slot: top row, bottom row, left column, right column
    has_halo = h < NH;
    if (h < TX) { hlx = h; hly = -1; }
    else if (h < 2 * TX) { hlx = h - TX; hly = TY; }
    else if (h < 2 * TX + RH) { hlx = -1; hly = h - 2 * TX - 1; }
    else { hlx = TX; hly = h - 2 * TX - RH - 1; }
    hx = wrapi(bx * TX + hlx, L.nx);
    hy = wrapi(by * TY + hly, L.ny);
    if (tid < CH) sm.chx[tid] = wrapi(bx * TX - E + tid * E, L.nx);
    cj = tid % CH;
    cr0 = tid < RS * CH ? tid / CH : NR;
  }

  // Row table of plane p (p in [-1, nz]).
  __device__ __forceinline__ void table(int p) {
    const int zp = wrapz(p);
    for (int R = threadIdx.x; R < NR; R += NT) {
      const int ci = R / RH, r = R - ci * RH, i = ci < Q ? ci : ci - Q;
      const int zs = wrapz(zp - dir_z_rt(i)), ys = wrap_near(y0 - 1 + r - dir_y_rt(i), L.ny);
      sm.rowp[R] = src + ((long long)ci * L.np + (long long)zs * L.nxny + (long long)ys * L.nx);
    }
  }

  // Copies of the plane whose table is current: this thread's chunk column cj of
  // rows cr0, cr0 + RS, ...; cx is that column's wrapped x.
  __device__ __forceinline__ void issue(int cx) {
    T* to = &sm.stage[0][0][0] + cr0 * SW + cj * E;
    constexpr int PASSES = (NR + RS - 1) / RS;  // rows cr0 + k RS < NR for every k < PASSES - 1
    if (cr0 < NR) {
#pragma unroll
      for (int k = 0; k < PASSES; ++k) {
        const int R = cr0 + k * RS;
        if (k < PASSES - 1 || R < NR) cp_async16(to + k * RS * SW, sm.rowp[R] + cx);
      }
    }
    cp_async_commit();
  }

  // Population i of component c arriving at tile cell (lx, ly) (ly, lx in [-1, TY] x [-1, TX]):
  // from the staged rows; next to a wall, a population whose source plane is solid
  // is the site's (index s) own opposite one instead.
  template <int I>
  __device__ __forceinline__ float staged(int c, int ly, int lx) const {
    return S::cv(sm.stage[c * Q + I][ly + 1][lx + E - dir_x(I)], wgt(I));
  }
  template <int I>
  __device__ __forceinline__ float pulled(int c, int ly, int lx, bool sol_m, bool sol_p, uint32_t s) const {
    constexpr int ez = dir_z(I);
    if (ez != 0 && (ez > 0 ? sol_m : sol_p))
      return S::ld(src + (long long)(c * Q + opp(I)) * L.np + s, wgt(I));
    return staged<I>(c, ly, lx);
  }

  // Read plane p out of the staged rows: the own site into fr/fb, the halo site
  // as sums (the owner's arithmetic, so the halo Psi has the owner's bits); apply the
  // sink and publish Psi to ring slot p & 3. Returns the own site's class.
  __device__ __forceinline__ int take(int p, bool own, float (&fr)[Q], float (&fb)[Q], float& rr, float& rb) {
    const int zp = wrapz(p), slot = p & 3;
    const bool sol_m = solid_z(L, zp == 0 ? L.nz - 1 : zp - 1), sol_p = solid_z(L, zp == L.nz - 1 ? 0 : zp + 1);
    const int cls = site_class(L, x, y, zp);
    float pr = 0.0f, pb = 0.0f;
    const bool walls = sol_m || sol_p;  // the same for the whole plane
    if (cls == SOLID) {
      rr = rb = 0.0f;
    } else {
      if (!walls) {
        Unroll<0, Q>::run([&](auto ic) {
          constexpr int I = decltype(ic)::value;
          fr[I] = staged<I>(0, ty, tx);
          fb[I] = staged<I>(1, ty, tx);
        });
      } else {
        const uint32_t s = (uint32_t)(x + L.nx * y) + (uint32_t)L.nxny * (uint32_t)zp;
        Unroll<0, Q>::run([&](auto ic) {
          constexpr int I = decltype(ic)::value;
          fr[I] = pulled<I>(0, ty, tx, sol_m, sol_p, s);
          fb[I] = pulled<I>(1, ty, tx, sol_m, sol_p, s);
        });
      }
      rr = sum19(fr);
      rb = sum19(fb);
      if (cls == SINK) {
        if (active && own && own_z(L, zp)) evap += (double)sink_excess(L, fr);
        sink_densities(L, rr, rb);
      }
      pr = psi_of(rr);
      pb = psi_of(rb);
    }
    sm.ring[slot][ty + 1][tx + 1] = make_float2(pr, pb);
    if (has_halo) {
      const int hcl = site_class(L, hx, hy, zp);
      float hpr = 0.0f, hpb = 0.0f;
      if (hcl != SOLID) {
        // the owner's arithmetic, so the halo Psi has the owner's bits
        float hrr, hrb;
        if (!walls) {
          hrr = sum19_of([&](auto ic) { return staged<decltype(ic)::value>(0, hly, hlx); });
          hrb = sum19_of([&](auto ic) { return staged<decltype(ic)::value>(1, hly, hlx); });
        } else {
          const uint32_t s = (uint32_t)(hx + L.nx * hy) + (uint32_t)L.nxny * (uint32_t)zp;
          hrr = sum19_of([&](auto ic) { return pulled<decltype(ic)::value>(0, hly, hlx, sol_m, sol_p, s); });
          hrb = sum19_of([&](auto ic) { return pulled<decltype(ic)::value>(1, hly, hlx, sol_m, sol_p, s); });
        }
        if (hcl == SINK) sink_densities(L, hrr, hrb);
        hpr = psi_of(hrr);
        hpb = psi_of(hrb);
      }
      sm.ring[slot][hly + 1][hlx + 1] = make_float2(hpr, hpb);
    }
    return cls;
  }

  // Collide plane z (in [0, nz); read out one plane earlier) and store f*.
  __device__ __forceinline__ void finish(int z, float (&fr)[Q], float (&fb)[Q], float rr, float rb, int cls) {
    if (!active || cls == SOLID) return;
    const int s = x + L.nx * y + L.nxny * z;
    if (cls == SINK) {
#pragma unroll
      for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, rr); fb[i] = rest_pop(i, rb); }
    } else {
      float ar[3], ab[3];
      auto psi2 = [&](int sl, int ly, int lx) { return sm.ring[sl][ly + 1][lx + 1]; };
      force_sums(psi2, (z - 1) & 3, z & 3, (z + 1) & 3, ty, tx, ar, ab);
      const float2 ps = sm.ring[z & 3][ty + 1][tx + 1];
      collide(L, fr, fb, rr, rb, ps.x, ps.y, ar, ab);
    }
    store_site<S>(L, dst, s, fr, fb);
  }

  __device__ __forceinline__ void run(int zb, int ze, bool down) {
    float cr[Q], cb[Q], nr[Q], nb[Q];
    float crr = 0.f, crb = 0.f, nrr = 0.f, nrb = 0.f;
    int ccl = SOLID;
    const int d = down ? -1 : 1;
    const int first = down ? ze - 1 : zb;
    const int n = ze - zb;
    table(first - d);
    __syncthreads();  // chunk and row tables
    const int cx = sm.chx[cj];
    issue(cx);
    for (int o = 0; o < n + 2; ++o) {
      const int p = first + (o - 1) * d;
      cp_async_wait_all();
      __syncthreads();  // every thread's copies of plane p have landed
      const int pcl = take(p, o >= 1 && o <= n, nr, nb, nrr, nrb);
      if (o + 1 < n + 2) table(p + d);
      __syncthreads();  // ring complete, staged rows read out, next table written
      if (o + 1 < n + 2) issue(cx);
      if (o >= 2) finish(p - d, cr, cb, crr, crb, ccl);
#pragma unroll
      for (int i = 0; i < Q; ++i) { cr[i] = nr[i]; cb[i] = nb[i]; }
      crr = nrr;
      crb = nrb;
      ccl = pcl;
    }
  }

  __device__ __forceinline__ double block_evap() {
    double v = evap;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
      for (int k = 0; k < NT / 32; ++k) t += sm.red[k];
    return t;
  }
};

// ------------------------------------------------------------------ in-place (AA) step
//
// One population lattice A updated in place. Between steps A holds, for every
// non-solid site x and direction i, the population arriving at x in direction i
// (the post-collision value of x - e_i, or x's own opposite one next to a wall):
//   even form: at (i, x - e_i), or at (opp(i), x) where x - e_i is solid -- the
//              slots the two-lattice pull reads (PullIdx::at);
//   odd form:  at (opp(i), x).
// A step reads the arrived populations of x and writes its post-collision f*_j
// into the slot that population opp(j) came from. In the even form that slot is
// where f*_j arrives in the odd form (x + e_j, or (j, x) when x + e_j is solid);
// in the odd form it is (j, x), the even form's slot of f*_j. The slots a site
// reads are exactly those it writes and belong to no other site, so no site's
// update touches another's data. Only the force couples sites: every neighbour's
// Psi must be formed before that neighbour is overwritten, so Psi comes from a
// separate pass (k_aa_psi) into an (Psi^r, Psi^b) array.

// Slot of the population arriving at the site of P in direction I.
template <int I, bool ODD>
__device__ __forceinline__ void aa_slot(const PullIdx& P, int& idx, int& d) {
  if (ODD) {
    idx = P.s;
    d = opp(I);
  } else {
    P.template at<I>(idx, d);
  }
}

// Arrived populations of the site of P (plain loads: the lattice is written in place).
template <class S, bool ODD>
__device__ __forceinline__ void aa_load(const LatDev& L, const typename S::T* A, const PullIdx& P, float (&fr)[Q],
                                        float (&fb)[Q]) {
  const long long cstride = (long long)Q * L.np;
  Unroll<0, Q>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int idx, d;
    aa_slot<I, ODD>(P, idx, d);
    const typename S::T* p = A + (long long)d * L.np + idx;
    fr[I] = S::cv(p[0], wgt(I));
    fb[I] = S::cv(p[cstride], wgt(I));
  });
}

// The same loads at L2 only (the persistent in-place step, where neighbouring CTAs
// rewrite slots this CTA read in an earlier step).
template <class S, bool ODD>
__device__ __forceinline__ void aa_load_cg(const LatDev& L, const typename S::T* A, const PullIdx& P, float (&fr)[Q],
                                           float (&fb)[Q]) {
  const long long cstride = (long long)Q * L.np;
  Unroll<0, Q>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int idx, d;
    aa_slot<I, ODD>(P, idx, d);
    const typename S::T* p = A + (long long)d * L.np + idx;
    fr[I] = S::ldcg(p, wgt(I));
    fb[I] = S::ldcg(p + cstride, wgt(I));
  });
}

// f*_j into the slot population opp(j) was read from.
template <class S, bool ODD>
__device__ __forceinline__ void aa_store(const LatDev& L, typename S::T* A, const PullIdx& P, const float (&fr)[Q],
                                         const float (&fb)[Q]) {
  const long long cstride = (long long)Q * L.np;
  Unroll<0, Q>::run([&](auto jc) {
    constexpr int J = decltype(jc)::value;
    int idx, d;
    aa_slot<opp(J), ODD>(P, idx, d);
    typename S::T* p = A + (long long)d * L.np + idx;
    S::st(p, fr[J], wgt(J));
    S::st(p + cstride, fb[J], wgt(J));
  });
}

}  // namespace sclbm
