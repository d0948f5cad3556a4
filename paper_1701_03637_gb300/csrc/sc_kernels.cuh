// Device code for the two-component Shan-Chen D3Q19 evaporation step
// (arXiv:1701.03637, Sec. II). Shared by the single-lattice and batched launches.
//
// State between launches ("pre-stream" form): the buffer holds post-collision
// populations f*(t-1). One launch pulls them (streaming with halfway
// bounce-back), applies the evaporation sink to the arrived populations, forms
// densities and Psi, the Eq. (3) force from a shared-memory Psi tile with a
// one-site halo, and collides (Eqs. (1), (2) with the tau F / rho velocity
// shift), writing f*(t) to the other buffer. The canonical (post-stream,
// post-sink) populations of step t are therefore pull + sink of the buffer.
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
  long long np;            // elements between consecutive direction arrays
  float omega[2], tau[2];  // 1/tau and tau per component
  float G, rhoH;           // g of Eq. (3); imposed rho^r at sinks
  double rhoH_mass;         // exact sum of the reset r populations fl(w_i rho_H)
  int geometry, sink_z0, sink_layers;
  double scx, scy, scz, RH2;
  int wall_z0, wall_z1;    // solid slab [wall_z0, wall_z1)
};

// ------------------------------------------------------------------ storage types
struct StF32 {
  using T = float;
  static __device__ __forceinline__ float ld(const T* p, float) { return __ldg(p); }
  static __device__ __forceinline__ void st(T* p, float v, float) { *p = v; }
};
// FP16 / BF16 offsets h = f - w_i * rho0 (rho0 = 1), round to nearest even.
struct StF16 {
  using T = __half;
  static __device__ __forceinline__ float ld(const T* p, float w) { return w + __half2float(__ldg(p)); }
  static __device__ __forceinline__ void st(T* p, float v, float w) { *p = __float2half_rn(v - w); }
};
struct StBF16 {
  using T = __nv_bfloat16;
  static __device__ __forceinline__ float ld(const T* p, float w) { return w + __bfloat162float(__ldg(p)); }
  static __device__ __forceinline__ void st(T* p, float v, float w) { *p = __float2bfloat16_rn(v - w); }
};

__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ bool solid_z(const LatDev& L, int z) { return z >= L.wall_z0 && z < L.wall_z1; }

// Site class from coordinates (no storage): solid slab, planar or spherical sink.
// The squared distance is formed without FMA contraction so it rounds the same
// way as a plain host evaluation.
__device__ __forceinline__ int site_class(const LatDev& L, int x, int y, int z) {
  if (solid_z(L, z)) return SOLID;
  if (L.geometry == 1) return wrapi(z - L.sink_z0, L.nz) < L.sink_layers ? SINK : FLUID;
  if (L.geometry == 2) {
    const double dx = (double)x - L.scx, dy = (double)y - L.scy, dz = (double)z - L.scz;
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
    return r2 >= L.RH2 ? SINK : FLUID;
  }
  return FLUID;
}

// Source offsets of the pull for site (x, y, z): the population arriving in
// direction i comes from x - e_i; from a solid site it is the site's own
// opposite population (halfway bounce-back).
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

// Same loads, summed in the same order as sum19() so both give identical bits.
template <class S>
__device__ __forceinline__ void pull_sums(const LatDev& L, const typename S::T* __restrict__ src, const PullIdx& P,
                                          float& rr, float& rb) {
  const long long cstride = (long long)Q * L.np;
  rr = 0.0f;
  rb = 0.0f;
  Unroll<0, Q>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int idx, d;
    P.template at<I>(idx, d);
    const typename S::T* p = src + (long long)d * L.np + idx;
    rr = rr + S::ld(p, wgt(I));
    rb = rb + S::ld(p + cstride, wgt(I));
  });
}

__device__ __forceinline__ float sum19(const float (&f)[Q]) {
  float r = 0.0f;
#pragma unroll
  for (int i = 0; i < Q; ++i) r = r + f[i];
  return r;
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

__device__ __forceinline__ float psi_of(float rho) { return 1.0f - expf(-rho); }  // Eq. (4), rho0 = 1

// Shifted-velocity BGK collision of one fluid site, storing f* (Eqs. (1)-(3)).
// ar/ab: sum_i w_i Psi^{r|b}(x + e_i) e_i.
template <class S>
__device__ __forceinline__ void collide_store(const LatDev& L, typename S::T* __restrict__ dst, int s,
                                              const float (&fr)[Q], const float (&fb)[Q], float rr, float rb,
                                              float psr, float psb, const float (&ar)[3], const float (&ab)[3]) {
  const float omr = L.omega[0], omb = L.omega[1];
  float mr[3] = {0.f, 0.f, 0.f}, mb[3] = {0.f, 0.f, 0.f};
  Unroll<1, Q>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    if (dir_x(I) > 0) { mr[0] += fr[I]; mb[0] += fb[I]; }
    if (dir_x(I) < 0) { mr[0] -= fr[I]; mb[0] -= fb[I]; }
    if (dir_y(I) > 0) { mr[1] += fr[I]; mb[1] += fb[I]; }
    if (dir_y(I) < 0) { mr[1] -= fr[I]; mb[1] -= fb[I]; }
    if (dir_z(I) > 0) { mr[2] += fr[I]; mb[2] += fb[I]; }
    if (dir_z(I) < 0) { mr[2] -= fr[I]; mb[2] -= fb[I]; }
  });
  const float den = rr * omr + rb * omb;
  const float inv = den > 0.0f ? 1.0f / den : 0.0f;
  float ur[3], ub[3];
  const float sr = rr > 0.0f ? L.tau[0] / rr : 0.0f;
  const float sb = rb > 0.0f ? L.tau[1] / rb : 0.0f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float up = (mr[d] * omr + mb[d] * omb) * inv;  // common velocity u'
    ur[d] = up + sr * (-L.G * psr * ab[d]);               // u' + tau F^r / rho^r
    ub[d] = up + sb * (-L.G * psb * ar[d]);               // u' + tau F^b / rho^b
  }
  const float usr = ur[0] * ur[0] + ur[1] * ur[1] + ur[2] * ur[2];
  const float usb = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
  const long long cstride = (long long)Q * L.np;
  // f^eq_i = w_i rho (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u.u); opposite directions share
  // the even part and differ in the sign of the odd part.
  {
    const float feqr = kW0 * rr * (1.0f - 1.5f * usr);
    const float feqb = kW0 * rb * (1.0f - 1.5f * usb);
    S::st(dst + s, fr[0] + omr * (feqr - fr[0]), kW0);
    S::st(dst + s + cstride, fb[0] + omb * (feqb - fb[0]), kW0);
  }
  Unroll<0, 9>::run([&](auto kc) {
    constexpr int I = 1 + 2 * decltype(kc)::value, J = I + 1;
    constexpr float w = wgt(I);
    const float cur = (float)dir_x(I) * ur[0] + (float)dir_y(I) * ur[1] + (float)dir_z(I) * ur[2];
    const float cub = (float)dir_x(I) * ub[0] + (float)dir_y(I) * ub[1] + (float)dir_z(I) * ub[2];
    const float wrr = w * rr, wrb = w * rb;
    const float evr = wrr * (1.0f + 4.5f * cur * cur - 1.5f * usr), odr = wrr * (3.0f * cur);
    const float evb = wrb * (1.0f + 4.5f * cub * cub - 1.5f * usb), odb = wrb * (3.0f * cub);
    typename S::T* pi = dst + (long long)I * L.np + s;
    typename S::T* pj = dst + (long long)J * L.np + s;
    S::st(pi, fr[I] + omr * ((evr + odr) - fr[I]), w);
    S::st(pj, fr[J] + omr * ((evr - odr) - fr[J]), w);
    S::st(pi + cstride, fb[I] + omb * ((evb + odb) - fb[I]), w);
    S::st(pj + cstride, fb[J] + omb * ((evb - odb) - fb[J]), w);
  });
}

template <class S>
__device__ __forceinline__ void store_plain(const LatDev& L, typename S::T* __restrict__ dst, int s,
                                            const float (&fr)[Q], const float (&fb)[Q]) {
  const long long cstride = (long long)Q * L.np;
#pragma unroll
  for (int i = 0; i < Q; ++i) {
    typename S::T* p = dst + (long long)i * L.np + s;
    S::st(p, fr[i], wgt(i));
    S::st(p + cstride, fb[i], wgt(i));
  }
}

// ------------------------------------------------------------------ fused step, one x-y tile column
//
// A CTA of TX*TY threads owns sites [x0, x0+TX) x [y0, y0+TY) and marches z over
// [zb, ze). Psi of the tile plus a one-site halo lives in a 4-plane shared ring,
// so the 18-neighbour force never reads Psi from HBM; halo densities are
// recomputed from the neighbours' pulled populations (an L2 hit when the
// neighbouring CTA is at the same plane). One barrier per plane: plane z+1 is
// written while plane z-2's slot is free.
template <int TX, int TY, class S>
struct Tile {
  static constexpr int NT = TX * TY, RW = TX + 2, RH = TY + 2, NH = 2 * TX + 2 * RH;
  static_assert(NH <= NT, "halo slots exceed threads");
  static_assert(NT % 32 == 0, "whole warps");

  struct Smem {
    float ring[2][4][RH][RW];
    double red[NT / 32];
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

  // Bind the CTA to tile column (bx, by).
  __device__ __forceinline__ void setup(int bx, int by) {
    const int tid = threadIdx.x;
    tx = tid % TX;
    ty = tid / TX;
    const int gx = bx * TX + tx, gy = by * TY + ty;
    active = gx < L.nx && gy < L.ny;
    x = gx % L.nx;
    y = gy % L.ny;
    has_halo = tid < NH;
    if (tid < TX) { hlx = tid; hly = -1; }
    else if (tid < 2 * TX) { hlx = tid - TX; hly = TY; }
    else if (tid < 2 * TX + RH) { hlx = -1; hly = tid - 2 * TX - 1; }
    else { hlx = TX; hly = tid - 2 * TX - RH - 1; }
    hx = wrapi(bx * TX + hlx, L.nx);
    hy = wrapi(by * TY + hly, L.ny);
  }

  // Pull plane p (the interior site into fr/fb, the halo slot as sums), apply
  // the sink, and publish Psi to ring slot p & 3.
  __device__ __forceinline__ void stage(int p, bool own, float (&fr)[Q], float (&fb)[Q], float& rr, float& rb,
                                        int& cls) {
    const int zp = wrapi(p, L.nz), slot = p & 3;
    cls = site_class(L, x, y, zp);
    float pr = 0.0f, pb = 0.0f;
    if (cls == SOLID) {
      rr = rb = 0.0f;
    } else {
      const PullIdx P(L, x, y, zp);
      pull_full<S>(L, src, P, fr, fb);
      rr = sum19(fr);
      rb = sum19(fb);
      if (cls == SINK) {
        if (active && own) evap += (double)sink_excess(L, fr);
        sink_densities(L, rr, rb);
      }
      pr = psi_of(rr);
      pb = psi_of(rb);
    }
    sm.ring[0][slot][ty + 1][tx + 1] = pr;
    sm.ring[1][slot][ty + 1][tx + 1] = pb;
    if (has_halo) {
      const int hc = site_class(L, hx, hy, zp);
      float hpr = 0.0f, hpb = 0.0f;
      if (hc != SOLID) {
        const PullIdx P(L, hx, hy, zp);
        float hrr, hrb;
        pull_sums<S>(L, src, P, hrr, hrb);
        if (hc == SINK) sink_densities(L, hrr, hrb);
        hpr = psi_of(hrr);
        hpb = psi_of(hrb);
      }
      sm.ring[0][slot][hly + 1][hlx + 1] = hpr;
      sm.ring[1][slot][hly + 1][hlx + 1] = hpb;
    }
  }

  // Collide plane z (values staged one plane earlier) and store f*.
  __device__ __forceinline__ void finish(int z, float (&fr)[Q], float (&fb)[Q], float rr, float rb, int cls) {
    if (!active || cls == SOLID) return;
    const int s = x + L.nx * y + L.nxny * z;
    if (cls == SINK) {
      // Sinks are neither forced nor collided: they stream f^eq(rho_H, 0) and
      // f^eq(rho^r + rho^b - rho_H, 0) as they are.
#pragma unroll
      for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, rr); fb[i] = rest_pop(i, rb); }
      store_plain<S>(L, dst, s, fr, fb);
      return;
    }
    const int s0 = z & 3, sm1 = (z - 1) & 3, sp1 = (z + 1) & 3;
    float ar[3] = {0.f, 0.f, 0.f}, ab[3] = {0.f, 0.f, 0.f};
    // opposite pairs (I, I+1): accumulate w_I (Psi(x+e_I) - Psi(x-e_I)) e_I
    Unroll<0, 9>::run([&](auto kc) {
      constexpr int I = 1 + 2 * decltype(kc)::value;
      constexpr int ex = dir_x(I), ey = dir_y(I), ez = dir_z(I);
      const int sa = ez > 0 ? sp1 : (ez < 0 ? sm1 : s0);
      const int sb = ez > 0 ? sm1 : (ez < 0 ? sp1 : s0);
      const float dr = sm.ring[0][sa][ty + 1 + ey][tx + 1 + ex] - sm.ring[0][sb][ty + 1 - ey][tx + 1 - ex];
      const float db = sm.ring[1][sa][ty + 1 + ey][tx + 1 + ex] - sm.ring[1][sb][ty + 1 - ey][tx + 1 - ex];
      constexpr float w = wgt(I);
      if (ex != 0) { ar[0] += (float)ex * (w * dr); ab[0] += (float)ex * (w * db); }
      if (ey != 0) { ar[1] += (float)ey * (w * dr); ab[1] += (float)ey * (w * db); }
      if (ez != 0) { ar[2] += (float)ez * (w * dr); ab[2] += (float)ez * (w * db); }
    });
    const float psr = sm.ring[0][s0][ty + 1][tx + 1], psb = sm.ring[1][s0][ty + 1][tx + 1];
    collide_store<S>(L, dst, s, fr, fb, rr, rb, psr, psb, ar, ab);
  }

  // March planes [zb, ze) upward (down = false) or downward. Each plane is staged
  // one plane ahead of its collision; the halo plane on the far side is staged
  // for Psi only.
  __device__ __forceinline__ void run(int zb, int ze, bool down) {
    float ar_[Q], ab_[Q], br_[Q], bb_[Q];
    float arr, arb, brr, brb;
    int acl, bcl;
    const int d = down ? -1 : 1;
    const int first = down ? ze - 1 : zb;
    const int n = ze - zb;
    auto own = [&](int p) { return p >= zb && p < ze; };
    stage(first - d, false, ar_, ab_, arr, arb, acl);
    stage(first, true, ar_, ab_, arr, arb, acl);
    for (int k = 0; k < n; k += 2) {
      const int z = first + d * k;
      stage(z + d, own(z + d), br_, bb_, brr, brb, bcl);
      __syncthreads();
      finish(z, ar_, ab_, arr, arb, acl);
      if (k + 1 >= n) break;
      stage(z + 2 * d, own(z + 2 * d), ar_, ab_, arr, arb, acl);
      __syncthreads();
      finish(z + d, br_, bb_, brr, brb, bcl);
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

}  // namespace sclbm
