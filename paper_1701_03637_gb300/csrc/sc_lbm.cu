// sc_lbm: C ABI and launches for the two-component Shan-Chen D3Q19 evaporation
// step on sm_103a (arXiv:1701.03637, Sec. II). include/sc_lbm.h documents the
// contract of every entry point.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "sc_kernels.cuh"
#include "sc_lbm.h"

using namespace sclbm;

namespace {

thread_local char g_err[512] = "no error";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess) return fail(SC_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

// Step kernel tile shapes (TX x TY sites per CTA).
constexpr int kNumTiles = 5;
constexpr int kTileX[kNumTiles] = {32, 32, 16, 8, 64};
constexpr int kTileY[kNumTiles] = {8, 4, 8, 4, 4};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// NVTX range over a host call of the C ABI, for Nsight timelines (a no-op when no
// tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }
int wrap_host(int v, int n) { return ((v % n) + n) % n; }

// ------------------------------------------------------------------ kernels

// Persistent fused step; Rows selects the staged-rows marcher (TileRows) over
// the per-thread one (Tile). CTA b marches items [starts[b], starts[b + 1]) of
// the host-built work list (see plan_launch): tile columns of TX x TY sites and
// z chunks, in every round the resident CTAs on neighbouring columns of the
// same chunk in lock-step, so that a column's halo and shifted-pull sectors are
// read from DRAM once and then from L2 by its neighbours.
template <int TX, int TY, class S, bool Rows>
__global__ void __launch_bounds__(TX * TY, (512 / (TX * TY)) > 1 ? 512 / (TX * TY) : 1)
    k_step(const LatDev L, const typename S::T* __restrict__ src, typename S::T* __restrict__ dst,
           double* __restrict__ evap_cum, int cols_x, const int4* __restrict__ items, const int* __restrict__ starts) {
  using TileT = std::conditional_t<Rows, TileRows<TX, TY, S>, Tile<TX, TY, S>>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<typename TileT::Smem*>(smem_raw);
  TileT t(L, sm, src, dst);
  const int i0 = starts[blockIdx.x], i1 = starts[blockIdx.x + 1];
  for (int it = i0; it < i1; ++it) {
    const int4 w = items[it];  // tile column, first plane, end plane, downward
    if (it > i0) __syncthreads();  // the previous item's last reads of the ring
    t.setup(w.x % cols_x, w.x / cols_x);
    t.run(w.y, w.z, w.w != 0);
  }
  if (L.geometry != 0) {
    const double e = t.block_evap();
    if (threadIdx.x == 0) evap_cum[blockIdx.x] += e;
  }
}

// ------------------------------------------------------------------ in-place (AA) step
//
// Each step is k_aa_psi then k_aa_collide, both persistent grids over row
// segments of kAAThreads sites (unit u: segment u % segs of row u / segs, row =
// y + ny z; CTA b takes units b, b + G, ...), so the resident CTAs work on
// neighbouring rows and the Psi rows of planes z - 1 .. z + 1 that a site's force
// reads are L2 hits after their first read. The arithmetic is the two-lattice
// step's (sum19, sink, psi_of, force_sums, collide), so the bits are the same.
constexpr int kAAThreads = 128;

struct AARow {
  int x, y, z;
  __device__ __forceinline__ AARow(const LatDev& L, long long u, int segs) {
    const long long row = u / segs;
    x = (int)(u - row * segs) * kAAThreads + (int)threadIdx.x;
    y = (int)(row % L.ny);
    z = (int)(row / L.ny);
  }
};

// (Psi^r, Psi^b) of every site from its arrived populations (after the sink
// reset of the densities); 0 at solid sites.
template <class S, bool ODD>
__global__ void __launch_bounds__(kAAThreads) k_aa_psi(const LatDev L, const typename S::T* A,
                                                       float2* __restrict__ psi, int segs, long long units) {
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const AARow r(L, u, segs);
    if (r.x >= L.nx) continue;
    const int cls = site_class(L, r.x, r.y, r.z);
    const PullIdx P(L, r.x, r.y, r.z);
    float2 v = make_float2(0.f, 0.f);
    if (cls != SOLID) {
      float fr[Q], fb[Q];
      aa_load<S, ODD>(L, A, P, fr, fb);
      float rr = sum19(fr), rb = sum19(fb);
      if (cls == SINK) sink_densities(L, rr, rb);
      v = make_float2(psi_of(rr), psi_of(rb));
    }
    psi[P.s] = v;
  }
}

// Stream (the arrived populations), sink, force from the Psi array, collision,
// and the in-place store of f*; each CTA adds its evaporated mass to its slot.
template <class S, bool ODD>
__global__ void __launch_bounds__(kAAThreads, 4) k_aa_collide(const LatDev L, typename S::T* A,
                                                              const float2* __restrict__ psi,
                                                              double* __restrict__ evap_cum, int segs,
                                                              long long units) {
  double evap = 0.0;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const AARow r(L, u, segs);
    if (r.x >= L.nx) continue;
    const int cls = site_class(L, r.x, r.y, r.z);
    if (cls == SOLID) continue;
    const PullIdx P(L, r.x, r.y, r.z);
    float fr[Q], fb[Q];
    aa_load<S, ODD>(L, A, P, fr, fb);
    float rr = sum19(fr), rb = sum19(fb);
    if (cls == SINK) {
      // neither forced nor collided: f^eq at rest of the reset densities
      evap += (double)sink_excess(L, fr);
      sink_densities(L, rr, rb);
#pragma unroll
      for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, rr); fb[i] = rest_pop(i, rb); }
    } else {
      const int nx = L.nx, ny = L.ny;
      auto psi2 = [&](int zb, int yy, int xx) {
        yy = yy < 0 ? yy + ny : (yy >= ny ? yy - ny : yy);
        xx = xx < 0 ? xx + nx : (xx >= nx ? xx - nx : xx);
        return psi[zb + yy * nx + xx];
      };
      float ar[3], ab[3];
      force_sums(psi2, P.zs[2], P.zs[1], P.zs[0], r.y, r.x, ar, ab);  // planes z - 1, z, z + 1
      const float2 ps = psi[P.s];
      collide(L, fr, fb, rr, rb, ps.x, ps.y, ar, ab);
    }
    aa_store<S, ODD>(L, A, P, fr, fb);
  }
  if (L.geometry != 0) {
    __shared__ double red[kAAThreads / 32];
    double v = evap;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int k = 0; k < kAAThreads / 32; ++k) t += red[k];
      evap_cum[blockIdx.x] += t;
    }
  }
}

// ------------------------------------------------------------------ persistent in-place (AA) step
//
// One cooperative launch advances K steps. The lattice is cut along x into B bands
// of equal width, marched one after another in every step (B = 1: the whole
// lattice at once). CTA k owns tile k of a cx x cy grid of TX x TY tiles over a
// band, in every band and every step, and marches its planes z = 0 .. nz-1: it
// forms Psi of plane p + 1 for its tile and a one-site halo ring (the halo from the
// neighbours' arrived populations) into a shared ring, then streams, applies the
// sink, forms the force and collides plane p and stores f* in place. Every
// population is read once by the Psi phase and once more by the collision, one
// plane later; the bands keep that second read an L2 hit on large planes (a plane
// of a 512^2 FP32 lattice is 40 MB, and three of them do not stay in the L2).
//
// What orders the CTAs: a site's arrived populations (its read set, which equals
// its write set) are overwritten only when its owner collides it, and a neighbour
// reads them (for its halo Psi) one plane earlier. So before colliding plane p a
// CTA waits until its 8 neighbours have formed Psi of plane p ("psi_done"), and
// before a band it waits until they have finished the previous band ("steps_done",
// one count per band). Both are 64-bit counters per CTA, released after a barrier
// and polled with acquire loads, tagged with the launch number in the high 32 bits.
// All CTAs are resident (cooperative launch), so the waits always end; each is still
// bounded by a time limit after which the CTA records where it gave up in `err` and
// returns (every other CTA then gives up too), and the host reports SC_ETIMEOUT.
// The planes nz - 1 (the halo below plane 0) and 0 (the halo above plane nz - 1) are
// formed first and kept in two extra ring slots, since both are rewritten before
// the march needs them again. Population loads bypass L1 (ld.global.cg): a line a
// CTA cached in one step may have been rewritten by a neighbour by the next.
//
// Band edges: when band b is marched, band b - 1 is finished (its populations
// overwritten) and band b + 1 not yet started (its populations still this step's
// arrived ones). So the halo column left of band b > 0 is Psi that band b - 1 saved
// from its last column, the halo right of band B - 1 is Psi that band 0 saved from
// its first column, and every other halo comes from the populations. The saved
// columns ("edge", [k][nz][ny]) are rewritten one step later, after every reader
// has finished the band that read them (the band count).
constexpr int kPersistMaxSteps = 1024;  // steps per launch (fewer when K B (nz + 2) would reach 2^32)
constexpr int kRingSlots = 6;           // rolling planes (4), plane nz - 1, plane 0 kept for the wrap

struct AAPersist {
  int cx, cy, TX, TY;           // tile grid over a band, and tile extents
  int B, bw;                    // bands along x, marched one after another, and their width
  int K, odd0;                  // steps of this launch; form of its first step
  unsigned long long epoch;     // launch number << 32
  unsigned long long* psi_done;    // [cx * cy]
  unsigned long long* steps_done;  // [cx * cy]: bands finished
  float2* edge;                 // saved Psi columns: [k][nz][ny], k = b for band b's last column
                                // (b < B - 1), k = B - 1 for band 0's first column
  int* err;                     // 0, or 1 + where a wait gave up
  long long limit_ns;           // wait limit
  int withhold;                 // this CTA never reports its Psi planes (-1: none): makes its
                                // neighbours' waits run out, to test the failure path
};

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Polled by threads 0..8 before a barrier: whether tile column (bx + dx, by + dy)
// (periodic; dx, dy in {-1, 0, 1} from the thread index, the CTA itself included)
// has counter >= target. False when the wait gave up (time limit, or another CTA
// gave up first); the first CTA to give up records `where` in the error word.
__device__ __forceinline__ bool poll_neighbour(const AAPersist& a, const unsigned long long* ctr,
                                               unsigned long long target, int bx, int by, int where) {
  const int dx = (int)threadIdx.x % 3 - 1, dy = (int)threadIdx.x / 3 - 1;
  const unsigned long long* p = ctr + (wrapi(bx + dx, a.cx) + a.cx * wrapi(by + dy, a.cy));
  if (ld_acquire_u64(p) >= target) return true;
  const unsigned long long t0 = global_ns();
  while (ld_acquire_u64(p) < target) {
    if (*(volatile int*)a.err != 0 || (long long)(global_ns() - t0) > a.limit_ns) {
      atomicCAS(a.err, 0, 1 + where);
      return false;
    }
  }
  return true;
}

template <class S, int NT>
struct PersistTile {
  using T = typename S::T;
  const LatDev& L;
  const AAPersist& a;
  T* A;
  float2* ring;
  int bx, by, band, x0, y0, tw, th, RW, cells;

  __device__ __forceinline__ int slot_of(int q) const {
    return (q == -1 || q == L.nz - 1) ? 4 : (q == L.nz ? 5 : (q & 3));
  }
  __device__ __forceinline__ float2& cell(int slot, int c) const { return ring[slot * cells + c]; }
  __device__ __forceinline__ float2* edge_at(int k, int z, int y) const {
    return a.edge + ((long long)k * L.nz + z) * L.ny + y;
  }

  // Psi of plane q (in [-1, nz]) over the tile and its halo ring into ring slot sa
  // (and sb >= 0); the 38 loads of a cell are independent and in flight together.
  // Ring cell c is site (x0 + hx, y0 + hy), hx = c % RW - 1, hy = c / RW - 1
  // (periodic); cells past a ragged tile's halo are skipped.
  template <bool ODD>
  __device__ __forceinline__ void psi_plane(int q, int sa, int sb) {
    const int zq = q < 0 ? q + L.nz : (q >= L.nz ? q - L.nz : q);
    const bool solid = solid_z(L, zq);
    const bool left_saved = a.B > 1 && bx == 0 && band > 0;               // band band - 1's last column
    const bool right_saved = a.B > 1 && bx == a.cx - 1 && band == a.B - 1;  // band 0's first column
    const bool save_last = a.B > 1 && bx == a.cx - 1 && band < a.B - 1;
    const bool save_first = a.B > 1 && bx == 0 && band == 0;
    for (int c = threadIdx.x; c < cells; c += NT) {
      const int hx = c % RW - 1, hy = c / RW - 1;
      if (hx > tw || hy > th) continue;
      const int x = wrap_near(x0 + hx, L.nx), y = wrap_near(y0 + hy, L.ny);
      float2 v = make_float2(0.f, 0.f);
      if (!solid) {
        if (hx == -1 && left_saved) {
          v = __ldcg(edge_at(band - 1, zq, y));
        } else if (hx == tw && right_saved) {
          v = __ldcg(edge_at(a.B - 1, zq, y));
        } else {
          float fr[Q], fb[Q];
          aa_load_cg<S, ODD>(L, A, PullIdx(L, x, y, zq), fr, fb);
          float rr = sum19(fr), rb = sum19(fb);
          if (site_class(L, x, y, zq) == SINK) sink_densities(L, rr, rb);
          v = make_float2(psi_of(rr), psi_of(rb));
        }
      }
      cell(sa, c) = v;
      if (sb >= 0) cell(sb, c) = v;
      if (hy >= 0 && hy < th) {
        if (save_last && hx == tw - 1) *edge_at(band, zq, y) = v;
        if (save_first && hx == 0) *edge_at(a.B - 1, zq, y) = v;
      }
    }
  }

  // Stream, sink, force, collision and in-place store of the tile's plane p.
  template <bool ODD>
  __device__ __forceinline__ void collide_plane(int p, double& evap) {
    const int sm1 = slot_of(p - 1), s0 = slot_of(p), sp1 = slot_of(p + 1);
    const int n = tw * th;
    for (int c = threadIdx.x; c < n; c += NT) {
      const int lx = c % tw, ly = c / tw;
      const int x = x0 + lx, y = y0 + ly;
      const int cls = site_class(L, x, y, p);
      if (cls == SOLID) continue;
      const PullIdx P(L, x, y, p);
      float fr[Q], fb[Q];
      aa_load_cg<S, ODD>(L, A, P, fr, fb);
      float rr = sum19(fr), rb = sum19(fb);
      if (cls == SINK) {
        evap += (double)sink_excess(L, fr);
        sink_densities(L, rr, rb);
#pragma unroll
        for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, rr); fb[i] = rest_pop(i, rb); }
      } else {
        auto psi2 = [&](int sl, int yy, int xx) { return cell(sl, (yy + 1) * RW + (xx + 1)); };
        float ar[3], ab[3];
        force_sums(psi2, sm1, s0, sp1, ly, lx, ar, ab);
        const float2 ps = cell(s0, (ly + 1) * RW + (lx + 1));
        collide(L, fr, fb, rr, rb, ps.x, ps.y, ar, ab);
      }
      aa_store<S, ODD>(L, A, P, fr, fb);
    }
  }

  // The march of one band in one step, one barrier per plane: the neighbours'
  // progress for the plane about to be written is polled before the Psi of the next
  // plane is formed, and the barrier after it both completes the ring and publishes
  // the poll; thread 0 then reports the new Psi plane. False when a wait gave up.
  template <bool ODD>
  __device__ __forceinline__ bool march(unsigned long long base, double& evap) {
    const int nz = L.nz;
    const bool reports = (int)blockIdx.x != a.withhold;
    psi_plane<ODD>(nz - 1, 4, -1);
    psi_plane<ODD>(0, 0, 5);
    __syncthreads();
    if (threadIdx.x == 0 && reports) st_release_u64(a.psi_done + blockIdx.x, base + 2);
    for (int p = 0; p < nz; ++p) {
      // every neighbour has formed Psi of plane p (read this tile's plane-p slots)
      const unsigned long long need = base + (p == nz - 1 ? 1ull : (p == 0 ? 2ull : (unsigned long long)(p + 2)));
      bool ok = true;
      if (threadIdx.x < 9) ok = poll_neighbour(a, a.psi_done, need, bx, by, 1);
      const bool more = p + 1 <= nz - 2;
      if (more) psi_plane<ODD>(p + 1, (p + 1) & 3, -1);
      if (__syncthreads_or(!ok)) return false;
      if (more && threadIdx.x == 0 && reports) st_release_u64(a.psi_done + blockIdx.x, base + (unsigned long long)(p + 3));
      collide_plane<ODD>(p, evap);
    }
    return true;
  }
};

// NT threads per CTA (128 or 256), 512 / NT CTAs per SM at 128 registers.
template <class S, int NT>
__global__ void __launch_bounds__(NT, 512 / NT)
    k_aa_persist(const LatDev L, typename S::T* A, double* __restrict__ evap_cum, const __grid_constant__ AAPersist a) {
  extern __shared__ __align__(16) float2 ring[];
  const int bx = (int)blockIdx.x % a.cx, by = (int)blockIdx.x / a.cx;
  PersistTile<S, NT> t{L, a, A, ring, bx, by, 0, 0, by * a.TY, 0, 0, a.TX + 2, (a.TX + 2) * (a.TY + 2)};
  t.tw = min(a.TX, a.bw - bx * a.TX);
  t.th = min(a.TY, L.ny - t.y0);
  double evap = 0.0;
  const unsigned long long per_band = (unsigned long long)L.nz + 2;
  bool ok = true;
  for (int s = 0; s < a.K && ok; ++s) {
    for (int b = 0; b < a.B && ok; ++b) {
      const unsigned long long sb = (unsigned long long)s * a.B + b;  // bands this launch marched before
      // the neighbours have finished the previous band (this band's populations are
      // their last writes; the saved edge columns are complete and read no more)
      if (sb > 0) {
        bool got = true;
        if (threadIdx.x < 9) got = poll_neighbour(a, a.steps_done, a.epoch + sb, bx, by, 0);
        if (__syncthreads_or(!got)) { ok = false; break; }
      }
      t.band = b;
      t.x0 = b * a.bw + bx * a.TX;
      const unsigned long long base = a.epoch + sb * per_band;
      ok = ((a.odd0 + s) & 1) ? t.template march<true>(base, evap) : t.template march<false>(base, evap);
      if (!ok) break;
      __syncthreads();  // every store and saved column of the band, then the report
      if (threadIdx.x == 0) st_release_u64(a.steps_done + blockIdx.x, a.epoch + sb + 1);
    }
  }
  if (L.geometry != 0) {
    __shared__ double red[NT / 32];
    double v = evap;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double tot = 0.0;
      for (int k = 0; k < NT / 32; ++k) tot += red[k];
      evap_cum[blockIdx.x] += tot;
    }
  }
}

// Arrived populations for the read-out kernels: the pull of the two-lattice
// buffer or of the in-place lattice's even form, or the odd form's own slots.
template <class S>
__device__ __forceinline__ void arrived(const LatDev& L, const typename S::T* __restrict__ src, const PullIdx& P,
                                        int odd, float (&fr)[Q], float (&fb)[Q]) {
  if (odd) aa_load<S, true>(L, src, P, fr, fb);
  else pull_full<S>(L, src, P, fr, fb);
}

__device__ __forceinline__ void site_of(const LatDev& L, long long s, int& x, int& y, int& z) {
  x = (int)(s % L.nx);
  y = (int)((s / L.nx) % L.ny);
  z = (int)(s / ((long long)L.nx * L.ny));
}

// Canonical state (pull + sink) of compact sites [s0, s1), as densities and/or
// populations in compact order.
template <class S>
__global__ void k_canonical(const LatDev L, const typename S::T* __restrict__ src, long long s0, long long s1,
                            float* __restrict__ rho_out, long long rho_stride, float* __restrict__ f_out,
                            long long f_stride, int odd) {
  for (long long s = s0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; s < s1;
       s += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    site_of(L, s, x, y, z);
    const int cls = site_class(L, x, y, z);
    float fr[Q], fb[Q], rr = 0.f, rb = 0.f;
    if (cls == SOLID) {
#pragma unroll
      for (int i = 0; i < Q; ++i) fr[i] = fb[i] = 0.f;
    } else {
      const PullIdx P(L, x, y, z);
      arrived<S>(L, src, P, odd, fr, fb);
      rr = sum19(fr);
      rb = sum19(fb);
      if (cls == SINK) {
        sink_densities(L, rr, rb);
#pragma unroll
        for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, rr); fb[i] = rest_pop(i, rb); }
      }
    }
    const long long o = s - s0;
    if (rho_out) { rho_out[o] = rr; rho_out[rho_stride + o] = rb; }
    if (f_out) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        f_out[(long long)i * f_stride + o] = fr[i];
        f_out[(long long)(Q + i) * f_stride + o] = fb[i];
      }
    }
  }
}

// FP64 plane diagnostics: per (plane, split) mass_r, mass_b, sum(rho_r - rho_b),
// pending evaporation of the canonical state, sites with rho_r > rho_b, flags.
constexpr int kDiagFields = 8;
constexpr int kDiagThreads = 256;

template <class S>
__global__ void __launch_bounds__(kDiagThreads) k_diag(const LatDev L, const typename S::T* __restrict__ src,
                                                       int nsplit, double* __restrict__ part, int odd) {
  const int z = blockIdx.x, k = blockIdx.y;
  const int nxy = L.nx * L.ny;
  const int per = (nxy + nsplit - 1) / nsplit;
  const int b = k * per, e = min(b + per, nxy);
  // mass_r, mass_b, sum(rho_r - rho_b), pending evaporation, count(rho_r > rho_b),
  // non-finite flag, negative-complement flag
  constexpr int NF = 7;
  double acc[NF] = {0, 0, 0, 0, 0, 0, 0};
  if (!solid_z(L, z) && own_z(L, z)) {  // a slab's ghost planes are not its own
    for (int q = b + threadIdx.x; q < e; q += blockDim.x) {
      const int x = q % L.nx, y = q / L.nx;
      const int cls = site_class(L, x, y, z);
      const PullIdx P(L, x, y, z);
      float fr[Q], fb[Q];
      arrived<S>(L, src, P, odd, fr, fb);
      float rr = sum19(fr), rb = sum19(fb);
      double mr = rr;
      if (cls == SINK) {
        acc[3] += (double)sink_excess(L, fr);
        sink_densities(L, rr, rb);
        mr = L.rhoH_mass;
        if (rb < 0.0f) acc[6] = 1.0;
      }
      if (!isfinite(rr) || !isfinite(rb)) acc[5] = 1.0;
      acc[0] += mr;
      acc[1] += rb;
      acc[2] += (double)rr - (double)rb;
      acc[4] += rr > rb ? 1.0 : 0.0;
    }
  }
  __shared__ double red[kDiagThreads / 32][NF];
#pragma unroll
  for (int j = 0; j < NF; ++j) {
    double v = acc[j];
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = (j >= 5) ? fmax(v, w) : v + w;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][j] = v;
  }
  __syncthreads();
  if (threadIdx.x < NF) {
    const int j = threadIdx.x;
    double t = 0.0;
    for (int w = 0; w < kDiagThreads / 32; ++w) t = (j >= 5) ? fmax(t, red[w][j]) : t + red[w][j];
    part[((long long)z * nsplit + k) * kDiagFields + j] = t;
  }
}

// ------------------------------------------------------------------ relative flux of Sec. III A
//
// j^r = rho^r (U^r - U) of Eqs. (flux) and (velw) (the paper states them for
// tau = 1): U = (m^r + m^b + (F^r + F^b) / 2) / (rho^r + rho^b) and U^r = (m^r + F^r
// + rho^r u') / (2 rho^r) with u' = (m^r + m^b) / (rho^r + rho^b) and F^c the force of
// Eq. (3) (periodic neighbours, Psi = 0 at solid sites, self couplings included),
// evaluated in FP64 from the canonical populations; 0 at sink and solid sites.
// Per (plane, split) partial sums of the three components go to `part`.

// FP64 densities of the canonical populations of site (x, y, z); returns its class.
template <class S>
__device__ __forceinline__ int canonical_rho(const LatDev& L, const typename S::T* __restrict__ src, int odd, int x,
                                             int y, int z, double& rr, double& rb, float (&fr)[Q], float (&fb)[Q]) {
  const int cls = site_class(L, x, y, z);
  rr = rb = 0.0;
  if (cls == SOLID) return cls;
  const PullIdx P(L, x, y, z);
  arrived<S>(L, src, P, odd, fr, fb);
  if (cls == SINK) {
    float a = sum19(fr), b = sum19(fb);
    sink_densities(L, a, b);
#pragma unroll
    for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, a); fb[i] = rest_pop(i, b); }
  }
#pragma unroll
  for (int i = 0; i < Q; ++i) { rr += (double)fr[i]; rb += (double)fb[i]; }
  return cls;
}

template <class S>
__global__ void __launch_bounds__(kDiagThreads) k_flux(const LatDev L, const typename S::T* __restrict__ src,
                                                       int nsplit, double* __restrict__ part, int odd, double G,
                                                       double g_rr, double g_bb) {
  const int z = blockIdx.x, k = blockIdx.y;
  const int nxy = L.nx * L.ny;
  const int per = (nxy + nsplit - 1) / nsplit;
  const int b = k * per, e = min(b + per, nxy);
  double acc[3] = {0.0, 0.0, 0.0};
  for (int q = b + threadIdx.x; q < e; q += blockDim.x) {
    const int x = q % L.nx, y = q / L.nx;
    float fr[Q], fb[Q];
    double rr, rb;
    if (canonical_rho<S>(L, src, odd, x, y, z, rr, rb, fr, fb) != FLUID) continue;
    double mr[3] = {0.0, 0.0, 0.0}, mb[3] = {0.0, 0.0, 0.0}, ar[3] = {0.0, 0.0, 0.0}, ab[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
      const double e[3] = {(double)dir_x(i), (double)dir_y(i), (double)dir_z(i)};
#pragma unroll
      for (int d = 0; d < 3; ++d) { mr[d] += e[d] * (double)fr[i]; mb[d] += e[d] * (double)fb[i]; }
    }
    // sum_i w_i Psi(x + e_i) e_i of both components over the 18 neighbours
#pragma unroll 1
    for (int i = 1; i < Q; ++i) {
      const int ex = dir_x(i), ey = dir_y(i), ez = dir_z(i);
      float gr[Q], gb[Q];
      double nr, nb;
      const int cls = canonical_rho<S>(L, src, odd, wrap_near(x + ex, L.nx), wrap_near(y + ey, L.ny),
                                       wrap_near(z + ez, L.nz), nr, nb, gr, gb);
      const double pr = cls == SOLID ? 0.0 : 1.0 - exp(-nr), pb = cls == SOLID ? 0.0 : 1.0 - exp(-nb);
      const double w = wgt_d(i);
      ar[0] += w * pr * ex; ar[1] += w * pr * ey; ar[2] += w * pr * ez;
      ab[0] += w * pb * ex; ab[1] += w * pb * ey; ab[2] += w * pb * ez;
    }
    const double psr = 1.0 - exp(-rr), psb = 1.0 - exp(-rb), rt = rr + rb;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      double Fr = -psr * G * ab[d], Fb = -psb * G * ar[d];
      if (g_rr != 0.0) Fr += -psr * g_rr * ar[d];
      if (g_bb != 0.0) Fb += -psb * g_bb * ab[d];
      if (rr > 0.0 && rt > 0.0) {
        const double U = (mr[d] + mb[d] + 0.5 * (Fr + Fb)) / rt;
        const double Ur = (mr[d] + Fr + rr * (mr[d] + mb[d]) / rt) / (2.0 * rr);
        acc[d] += rr * (Ur - U);
      }
    }
  }
  __shared__ double red[kDiagThreads / 32][3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double v = acc[d];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][d] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < kDiagThreads / 32; ++w) t += red[w][threadIdx.x];
    part[((long long)z * nsplit + k) * kDiagFields + threadIdx.x] = t;
  }
}

// ------------------------------------------------------------------ diagnostics without allocation
//
// For callers that cannot allocate device memory: the per-plane partial sums
// of k_diag go to this file-scope array (every device that loads the library
// holds it until the process exits) instead of the handle's buffer, and
// k_diag_finish folds them on the device, in the host reduction's order, into
// the caller's output. k_diag overwrites every slot a call reads, so nothing
// carries over between calls; calls that overlap on the GPU share the array and
// race.
constexpr long long kNoAllocScratch = 262144;  // doubles, 2 MiB per device
__device__ __align__(256) double g_noalloc_scratch[kNoAllocScratch];

__global__ void k_diag_finish(const double* __restrict__ part, int nz, int nsplit, double nxy, int wall_z0,
                              int wall_z1, const double* __restrict__ evap_slots, long long nslots,
                              double evap_offset, const int* __restrict__ persist_err, double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double mass_r = 0.0, mass_b = 0.0, pending = 0.0, count = 0.0, nonfinite = 0.0, sinkneg = 0.0;
  const int z0 = wall_z1 > wall_z0 ? wall_z1 : 0;
  double interface_z = -1.0, prev = 0.0;
  bool have_prev = false;
  for (int z = 0; z < nz; ++z) {
    double pz = 0.0;
    for (int k = 0; k < nsplit; ++k) {
      const double* q = part + ((long long)z * nsplit + k) * kDiagFields;
      mass_r += q[0];
      mass_b += q[1];
      pz += q[2];
      pending += q[3];
      count += q[4];
      nonfinite = fmax(nonfinite, q[5]);
      sinkneg = fmax(sinkneg, q[6]);
    }
    const bool solid = wall_z0 <= z && z < wall_z1;
    const double phi = pz / nxy;
    // first downward zero crossing of phi above the liquid base
    if (interface_z < 0.0 && have_prev && z - 1 >= z0 && prev > 0.0 && phi <= 0.0 && !solid)
      interface_z = (z - 1) + prev / (prev - phi);
    have_prev = !solid;
    prev = phi;
  }
  double cum = 0.0;
  for (long long k = 0; k < nslots; ++k) cum += evap_slots[k];
  out[0] = mass_r;
  out[1] = mass_b;
  out[2] = evap_offset + cum + pending;
  out[3] = pending;
  out[4] = interface_z;
  out[5] = cbrt(3.0 * count / (4.0 * 3.141592653589793));
  out[6] = count;
  const bool bad = nonfinite > 0.0 || !isfinite(mass_r) || !isfinite(mass_b);
  out[7] = bad ? (double)SC_ENONFINITE : (sinkneg > 0.0 ? (double)SC_ESINKNEG : (double)SC_OK);
  if (persist_err && *persist_err != 0) out[7] = (double)SC_ETIMEOUT;
}

// Initial / restored state: canonical populations of sites [s0, s1) from
// (mode 0) an FP32 population slab, (mode 1) density fields, (mode 2) the seeded
// film/droplet shape. Sinks are reset (evaporated mass not counted) and each
// value is written to the slot the next pull of that site reads it from.
struct ShapeDev {
  int shape, film_z;
  double cx, cy, cz, R2, hi, lo, amp;
  unsigned long long seed;
};

// SplitMix64 (Steele, Lea & Flood 2014): output k of the generator seeded with
// `seed` is the finaliser applied to seed + k * 0x9E3779B97F4A7C15.
__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + k * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

template <class S>
__global__ void k_load(const LatDev L, typename S::T* __restrict__ dst, long long s0, long long s1, int mode,
                       const float* __restrict__ f_in, long long f_stride, const float* __restrict__ rho_in,
                       long long rho_stride, const ShapeDev sh, long long nsites) {
  for (long long s = s0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; s < s1;
       s += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    site_of(L, s, x, y, z);
    const int cls = site_class(L, x, y, z);
    if (cls == SOLID) continue;
    const long long o = s - s0;
    float fr[Q], fb[Q];
    if (mode == 0) {
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fr[i] = f_in[(long long)i * f_stride + o];
        fb[i] = f_in[(long long)(Q + i) * f_stride + o];
      }
    } else if (mode == 1) {
      const float r = rho_in[o], b = rho_in[rho_stride + o];
#pragma unroll
      for (int i = 0; i < Q; ++i) { fr[i] = wgt(i) * r; fb[i] = wgt(i) * b; }
    } else {
      bool rich;
      const int zg = global_z(L, z);  // the shape and the noise are the whole lattice's
      const long long sg = (long long)x + (long long)L.nx * ((long long)y + (long long)L.ny * zg);
      if (sh.shape == 0) {
        rich = zg < sh.film_z;
      } else {
        const double dx = (double)x - sh.cx, dy = (double)y - sh.cy, dz = (double)zg - sh.cz;
        rich = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) < sh.R2;
      }
      const double ur = (double)(splitmix64_at(sh.seed, 1ULL + (unsigned long long)sg) >> 11) * 0x1.0p-53;
      const double ub =
          (double)(splitmix64_at(sh.seed, 1ULL + (unsigned long long)nsites + (unsigned long long)sg) >> 11) * 0x1.0p-53;
      const double r = (rich ? sh.hi : sh.lo) + __dmul_rn(sh.amp, __dadd_rn(2.0 * ur, -1.0));
      const double b = (rich ? sh.lo : sh.hi) + __dmul_rn(sh.amp, __dadd_rn(2.0 * ub, -1.0));
#pragma unroll
      for (int i = 0; i < Q; ++i) {
        fr[i] = (float)__dmul_rn(wgt_d(i), r);
        fb[i] = (float)__dmul_rn(wgt_d(i), b);
      }
    }
    if (cls == SINK) {
      float rr = sum19(fr), rb = sum19(fb);
      sink_densities(L, rr, rb);
#pragma unroll
      for (int i = 0; i < Q; ++i) { fr[i] = rest_pop(i, rr); fb[i] = rest_pop(i, rb); }
    }
    // inverse of the pull: f_i(x) is read from x - e_i (wrapped), or from (x, opp(i))
    // when plane z - e_iz is solid.
    const long long cstride = (long long)Q * L.np;
    Unroll<0, Q>::run([&](auto ic) {
      constexpr int I = decltype(ic)::value;
      const int zs = wrapi(z - dir_z(I), L.nz);
      const bool sol = dir_z(I) != 0 && solid_z(L, zs);
      const int idx = sol ? x + L.nx * y + L.nxny * z
                          : wrapi(x - dir_x(I), L.nx) + L.nx * wrapi(y - dir_y(I), L.ny) + L.nxny * zs;
      const int d = sol ? opp(I) : I;
      typename S::T* p = dst + (long long)d * L.np + idx;
      S::st(p, fr[I], wgt(I));
      S::st(p + cstride, fb[I], wgt(I));
    });
  }
}

// ------------------------------------------------------------------ launch tables

struct StepArgs {
  LatDev L;
  const void* src;
  void* dst;
  double* evap;
  int cols_x;
  const int4* items;
  const int* starts;
  int G;
  cudaStream_t st;
};

template <int TX, int TY, class S, bool Rows = false>
constexpr size_t step_smem() {
  return Rows ? sizeof(typename TileRows<TX, TY, S>::Smem) : sizeof(typename Tile<TX, TY, S>::Smem);
}

template <int TX, int TY, class S, bool Rows>
cudaError_t launch_step(const StepArgs& a) {
  k_step<TX, TY, S, Rows><<<a.G, TX * TY, step_smem<TX, TY, S, Rows>(), a.st>>>(
      a.L, (const typename S::T*)a.src, (typename S::T*)a.dst, a.evap, a.cols_x, a.items, a.starts);
  return cudaGetLastError();
}

// Resident CTAs per SM on the current device. Also opts the kernel in to its
// dynamic shared memory there (above the 48 KB default); every handle calls this
// on its device before its first step.
template <int TX, int TY, class S, bool Rows>
int occupancy_step() {
  int nb = 0;
  if (cudaFuncSetAttribute(k_step<TX, TY, S, Rows>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_smem<TX, TY, S, Rows>()) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_step<TX, TY, S, Rows>, TX * TY,
                                                    step_smem<TX, TY, S, Rows>()) != cudaSuccess)
    return 0;
  return nb;
}

using LaunchFn = cudaError_t (*)(const StepArgs&);
struct StepOps {
  LaunchFn launch;
  int (*occupancy)();  // resident CTAs per SM
};

template <class S, bool Rows>
StepOps pick_step(int tile) {
  switch (tile) {
    case 0: return {&launch_step<32, 8, S, Rows>, &occupancy_step<32, 8, S, Rows>};
    case 1: return {&launch_step<32, 4, S, Rows>, &occupancy_step<32, 4, S, Rows>};
    case 2: return {&launch_step<16, 8, S, Rows>, &occupancy_step<16, 8, S, Rows>};
    case 4: return {&launch_step<64, 4, S, Rows>, &occupancy_step<64, 4, S, Rows>};
    default: return {&launch_step<8, 4, S, Rows>, &occupancy_step<8, 4, S, Rows>};
  }
}

StepOps step_ops(int storage, int tile, bool rows) {
  switch (storage) {
    case SC_STORAGE_F16: return rows ? pick_step<StF16, true>(tile) : pick_step<StF16, false>(tile);
    case SC_STORAGE_F16_SCALED: return rows ? pick_step<StF16S, true>(tile) : pick_step<StF16S, false>(tile);
    case SC_STORAGE_BF16: return rows ? pick_step<StBF16, true>(tile) : pick_step<StBF16, false>(tile);
    default: return rows ? pick_step<StF32, true>(tile) : pick_step<StF32, false>(tile);
  }
}

constexpr long long kMaxCtas = 4096;  // evaporated-mass slots, one per CTA of the persistent step
constexpr int kSlabGhosts = 2;        // ghost planes on each side of a z-slab

size_t elem_size(int storage) { return storage == SC_STORAGE_F32 ? 4 : 2; }

struct Layout {
  int tile, tx, ty, cols_x, cols;
  bool rows;                  // staged-rows step kernel (nx a multiple of a 16-byte chunk)
  bool aa;                    // one population lattice updated in place (SC_LAYOUT_AA)
  int aa_segs;                // row segments of kAAThreads sites per row (in place)
  long long aa_units;         // row segments of the lattice (in place)
  long long np;               // array stride (elements)
  long long nsites, stage_n;  // sites; staging floats per component
  long long units, nslots;
  int diag_nsplit;
  long long cap_items;         // work-list capacity (items of any tile shape and schedule)
  size_t off_pop[2], off_psi, off_stage, off_evap, off_diag, off_items, off_starts, off_flags, total;
};

int auto_tile(const sc_params* p) {
  if (p->nx >= 32) return p->ny >= 8 ? 0 : 1;
  if (p->nx >= 16) return 2;
  return 3;
}

Layout make_layout(const sc_params* p) {
  Layout l{};
  const long long es = (long long)elem_size(p->storage);
  l.tile = p->tile > 0 ? p->tile - 1 : auto_tile(p);
  l.tx = kTileX[l.tile];
  l.ty = kTileY[l.tile];
  l.aa = p->layout == SC_LAYOUT_AA;
  l.rows = !l.aa && (p->staging == SC_STAGING_ROWS || (p->staging == SC_STAGING_AUTO && p->nx % (16 / es) == 0));
  l.nsites = (long long)p->nx * p->ny * p->nz;
  l.np = round_up(l.nsites, 128 / es);  // each array starts 128-byte aligned
  l.stage_n = round_up(l.nsites, 64);
  l.cols_x = (p->nx + l.tx - 1) / l.tx;
  l.cols = l.cols_x * ((p->ny + l.ty - 1) / l.ty);
  l.units = (long long)l.cols * p->nz;
  l.aa_segs = (p->nx + kAAThreads - 1) / kAAThreads;
  l.aa_units = (long long)l.aa_segs * p->ny * p->nz;
  // evaporated-mass slots: one per CTA of the persistent step (at most kMaxCtas),
  // and at least one per tile column of the smallest tile, so that a batch, which
  // books every (tile column, z chunk) item in a slot of its own, never has more
  // items of this lattice than slots (member_nch in sc_batch.cuh)
  const long long min_tile_cols = (long long)((p->nx + 7) / 8) * ((p->ny + 3) / 4);
  l.nslots = std::max(std::min(l.aa ? l.aa_units : l.units, kMaxCtas), min_tile_cols);
  const long long per_plane = (long long)p->nx * p->ny;
  l.diag_nsplit = (int)std::max(1LL, std::min<long long>((4LL * 152 + p->nz - 1) / p->nz, (per_plane + 1023) / 1024));
  const size_t pop = align256((size_t)(2 * Q * l.np * es));
  size_t off = 0;
  l.off_pop[0] = off; off += pop;
  l.off_pop[1] = l.off_pop[0];
  l.off_psi = off;
  if (l.aa) off += align256((size_t)l.np * sizeof(float2));  // (Psi^r, Psi^b) per site
  else { l.off_pop[1] = off; off += pop; }
  l.off_stage = off; off += align256((size_t)2 * l.stage_n * sizeof(float));
  l.off_evap = off; off += align256((size_t)l.nslots * sizeof(double));
  l.off_diag = off; off += align256((size_t)p->nz * l.diag_nsplit * kDiagFields * sizeof(double));
  // work list: at most one item per (column of the smallest tile, plane), plus one
  // split per CTA of the balanced schedule (under 1 byte per site)
  l.cap_items = (long long)((p->nx + 7) / 8) * ((p->ny + 3) / 4) * p->nz + kMaxCtas;
  l.off_items = off; off += align256((size_t)l.cap_items * sizeof(int4));
  l.off_starts = off; off += align256((size_t)(kMaxCtas + 1) * sizeof(int));
  // progress counters of the persistent in-place step (two per CTA) and its error word
  l.off_flags = off; off += align256((size_t)2 * kMaxCtas * sizeof(unsigned long long) + 256);
  l.total = off;
  return l;
}

int validate(const sc_params* p) {
  if (!p) return fail(SC_EINVAL, "params is NULL");
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(SC_EINVAL, "lattice extents must be >= 1");
  if (!(p->tau_r > 0.5) || !(p->tau_b > 0.5) || !std::isfinite(p->tau_r) || !std::isfinite(p->tau_b))
    return fail(SC_EINVAL, "tau must exceed 1/2");
  if (!std::isfinite(p->G) || !std::isfinite(p->rho_H)) return fail(SC_EINVAL, "G and rho_H must be finite");
  if (!std::isfinite(p->G_rr) || !std::isfinite(p->G_bb)) return fail(SC_EINVAL, "self couplings must be finite");
  if (p->geometry < 0 || p->geometry > 2) return fail(SC_EINVAL, "unknown geometry %d", p->geometry);
  if (p->geometry == 1 && (p->sink_layers < 1 || p->sink_layers > p->nz))
    return fail(SC_EINVAL, "sink_layers must be in [1, nz]");
  if (p->geometry == 2 && !(p->R_H > 0)) return fail(SC_EINVAL, "R_H must be > 0");
  if (p->wall_thickness < 0 || (p->wall_thickness > 0 && (p->wall_z0 < 0 || p->wall_z0 + p->wall_thickness > p->nz)))
    return fail(SC_EINVAL, "wall slab must lie inside [0, nz)");
  if (p->storage < 0 || p->storage > 3) return fail(SC_EINVAL, "unknown storage %d", p->storage);
  if (p->tile < 0 || p->tile > kNumTiles) return fail(SC_EINVAL, "tile index out of range");
  if (p->zchunk < 0) return fail(SC_EINVAL, "zchunk must be >= 0");
  if (p->staging < SC_STAGING_AUTO || p->staging > SC_STAGING_PERSISTENT) return fail(SC_EINVAL, "unknown staging %d", p->staging);
  if (p->staging == SC_STAGING_PERSISTENT && p->layout != SC_LAYOUT_AA)
    return fail(SC_EINVAL, "the persistent step is an in-place step (layout SC_LAYOUT_AA)");
  if (p->layout != SC_LAYOUT_TWO_LATTICE && p->layout != SC_LAYOUT_AA) return fail(SC_EINVAL, "unknown layout %d", p->layout);
  if (p->staging == SC_STAGING_ROWS && p->nx % (p->storage == SC_STORAGE_F32 ? 4 : 8) != 0)
    return fail(SC_EINVAL, "staged rows need nx to be a multiple of %d", p->storage == SC_STORAGE_F32 ? 4 : 8);
  if ((long long)p->nx > (1 << 20) || (long long)p->ny > (1 << 20) || (long long)p->nz > (1 << 20))
    return fail(SC_EINVAL, "lattice extent too large");
  if ((long long)p->nx * p->ny * p->nz > (1LL << 31) - 4096)
    return fail(SC_EINVAL, "lattice too large: nx*ny*nz must stay below 2^31");
  return SC_OK;
}

LatDev make_dev(const sc_params* p, const Layout& l) {
  LatDev L{};
  L.nx = p->nx; L.ny = p->ny; L.nz = p->nz; L.nxny = p->nx * p->ny;
  L.np = l.np;
  L.tau[0] = (float)p->tau_r; L.tau[1] = (float)p->tau_b;
  L.omega[0] = (float)(1.0 / p->tau_r); L.omega[1] = (float)(1.0 / p->tau_b);
  L.G = (float)p->G;
  L.Gs[0] = (float)p->G_rr;
  L.Gs[1] = (float)p->G_bb;
  L.rhoH = (float)p->rho_H;
  L.rhoH_mass = 0.0;
  for (int i = 0; i < Q; ++i) L.rhoH_mass += (double)(wgt(i) * (float)p->rho_H);
  L.geometry = p->geometry;
  L.sink_z0 = wrap_host(p->sink_z0, p->nz); L.sink_layers = p->sink_layers;
  L.scx = p->sphere_cx; L.scy = p->sphere_cy; L.scz = p->sphere_cz; L.RH2 = p->R_H * p->R_H;
  if (p->wall_thickness > 0) { L.wall_z0 = p->wall_z0; L.wall_z1 = p->wall_z0 + p->wall_thickness; }
  else { L.wall_z0 = 0; L.wall_z1 = 0; }
  L.zoff = 0;
  L.nzg = p->nz;
  L.own0 = 0;
  L.own1 = p->nz;
  return L;
}

}  // namespace

struct sc_lbm {
  sc_params p;
  Layout lay;
  LatDev L;
  cudaStream_t stream;
  char* base;
  bool owns;
  int cur;  // buffer holding the current pre-stream state
  int64_t step;
  double evap_offset;  // evaporated mass restored by sc_lbm_set_counters
  double* h_diag;      // pinned
  double* h_evap;      // pinned
  int grid;  // CTAs of the persistent step (in place: of k_aa_collide)
  int grid_psi;  // CTAs of k_aa_psi
  // persistent in-place step (k_aa_persist), when the layout is in place and it fits
  bool persist;
  int pcx, pcy, ptx, pty;    // its tile grid over a band and tile extents (grid = pcx * pcy CTAs)
  int pband;                 // bands along x, marched one after another
  int pband_req;             // requested band count (0: automatic)
  int pnt;                   // its threads per CTA
  size_t psmem;              // its dynamic shared memory
  unsigned launch_no;        // launches so far (tags the progress counters)
  long long wait_limit_ns;   // limit of each of its waits
  int withhold;              // CTA that withholds its progress reports (-1: none)
  const char* persist_why;   // why the persistent step was not planned
  bool slab;                 // z-slab of a larger lattice (sc_slab_create)
  int zmax;  // planes of the longest work item
  cudaGraphExec_t graph;
  int graph_len;
  int graph_cur;
  sc_batch* owner;  // batch whose arena holds this lattice (it destroys the handle)
  void* pop(int k) const { return base + lay.off_pop[k]; }
  float2* psi() const { return (float2*)(base + lay.off_psi); }
  int odd() const { return lay.aa && cur == 1 ? 1 : 0; }  // in-place lattice in its odd form
  float* stage() const { return (float*)(base + lay.off_stage); }
  double* evap() const { return (double*)(base + lay.off_evap); }
  double* diag() const { return (double*)(base + lay.off_diag); }
  int4* items() const { return (int4*)(base + lay.off_items); }
  int* starts() const { return (int*)(base + lay.off_starts); }
  unsigned long long* flags() const { return (unsigned long long*)(base + lay.off_flags); }
  int* err() const { return (int*)(base + lay.off_flags + 2 * kMaxCtas * sizeof(unsigned long long)); }
};

namespace {

// Launch configuration of the persistent step for one tile shape: the grid and
// the work list, CTA b taking items [starts[b], starts[b + 1]).
struct LaunchCfg {
  int tile, cols_x, cols, grid, zmax;
  std::vector<int4> items;  // tile column, first plane, end plane, downward
  std::vector<int> starts;
};

// Plans the persistent grid (every resident CTA slot, at most the handle's
// evaporated-mass slots) and its chunk-major work list: z is cut into nch
// chunks, item i = (chunk i / cols, column i % cols), CTA b taking items b,
// b + G, ...; in each round the resident CTAs work on neighbouring columns of
// the same chunk in lock-step, so a column's halo and shifted-pull sectors come
// from L2 for its neighbours. Chunks alternate their marching direction. The
// chunk count trades rounds (ceil(items / G)) against the two halo planes each
// item stages; zchunk > 0 fixes the chunk length instead.
int plan_launch(const sc_params* p, const Layout& l, int tile, int zchunk, LaunchCfg* c) {
  int dev = 0, sms = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int occ = step_ops(p->storage, tile, l.rows).occupancy();
  if (occ < 1) return fail(SC_ECUDA, "the step kernel cannot be made resident: %s", cudaGetErrorString(cudaGetLastError()));
  c->tile = tile;
  c->cols_x = (p->nx + kTileX[tile] - 1) / kTileX[tile];
  c->cols = c->cols_x * ((p->ny + kTileY[tile] - 1) / kTileY[tile]);
  const long long slots = std::min<long long>((long long)sms * occ, l.nslots), cols = c->cols, nz = p->nz;
  long long best_nch = 1;
  if (zchunk > 0) {
    best_nch = (nz + zchunk - 1) / zchunk;
  } else {
    double best = 1e300;
    for (long long nch = 1; nch <= nz && cols * nch <= l.cap_items; ++nch) {
      const long long rounds = (cols * nch + slots - 1) / slots;
      const double cost = (double)rounds * ((double)((nz + nch - 1) / nch) + 2.0);
      if (cost < best * (1.0 - 1e-9)) { best = cost; best_nch = nch; }
    }
  }
  const long long n = cols * best_nch;
  if (n > l.cap_items) return fail(SC_EINVAL, "work list exceeds its capacity");
  c->grid = (int)std::max(1LL, std::min<long long>(slots, n));
  c->items.clear();
  c->starts.clear();
  c->zmax = 0;
  for (long long b = 0; b < c->grid; ++b) {
    c->starts.push_back((int)c->items.size());
    for (long long it = b; it < n; it += c->grid) {
      const long long k = it / cols, col = it - k * cols;
      const int zb = (int)(k * nz / best_nch), ze = (int)((k + 1) * nz / best_nch);
      c->items.push_back(make_int4((int)col, zb, ze, (int)(k & 1)));
      c->zmax = std::max(c->zmax, ze - zb);
    }
  }
  c->starts.push_back((int)c->items.size());
  return SC_OK;
}

// Makes c the handle's configuration and uploads its work list (synchronous).
int apply_launch(sc_lbm* h, const LaunchCfg& c) {
  CK(cudaMemcpyAsync(h->items(), c.items.data(), sizeof(int4) * c.items.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(h->starts(), c.starts.data(), sizeof(int) * c.starts.size(), cudaMemcpyHostToDevice, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->lay.tile = c.tile;
  h->lay.tx = kTileX[c.tile];
  h->lay.ty = kTileY[c.tile];
  h->lay.cols_x = c.cols_x;
  h->lay.cols = c.cols;
  h->zmax = c.zmax;
  h->grid = c.grid;
  return SC_OK;
}

// In-place step launches for one storage type.
template <class S>
cudaError_t launch_aa(const sc_lbm* h, cudaStream_t st) {
  using T = typename S::T;
  const Layout& l = h->lay;
  if (h->cur == 1) {
    k_aa_psi<S, true><<<h->grid_psi, kAAThreads, 0, st>>>(h->L, (const T*)h->pop(0), h->psi(), l.aa_segs, l.aa_units);
    k_aa_collide<S, true><<<h->grid, kAAThreads, 0, st>>>(h->L, (T*)h->pop(0), h->psi(), h->evap(), l.aa_segs,
                                                          l.aa_units);
  } else {
    k_aa_psi<S, false><<<h->grid_psi, kAAThreads, 0, st>>>(h->L, (const T*)h->pop(0), h->psi(), l.aa_segs, l.aa_units);
    k_aa_collide<S, false><<<h->grid, kAAThreads, 0, st>>>(h->L, (T*)h->pop(0), h->psi(), h->evap(), l.aa_segs,
                                                           l.aa_units);
  }
  return cudaGetLastError();
}

template <class S>
void occupancy_aa(int* psi_occ, int* collide_occ) {
  int a = 0, b = 0, c = 0, d = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_aa_psi<S, false>, kAAThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_aa_psi<S, true>, kAAThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_aa_collide<S, false>, kAAThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_aa_collide<S, true>, kAAThreads, 0);
  *psi_occ = std::min(a, b);
  *collide_occ = std::min(c, d);
}

bool plan_persist(sc_lbm* h);

// The handle's launch description after a persistent plan.
void apply_persist(sc_lbm* h) {
  h->grid = h->pcx * h->pcy;
  h->zmax = h->p.nz;
  h->lay.tx = h->ptx;
  h->lay.ty = h->pty;
  if (h->withhold >= h->grid) h->withhold = -1;
}

// Grids of the in-place step: every resident CTA slot, the collision's at most
// the evaporated-mass slots.
int plan_aa(sc_lbm* h) {
  int dev = 0, sms = 1, po = 0, co = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  switch (h->p.storage) {
    case SC_STORAGE_F16: occupancy_aa<StF16>(&po, &co); break;
    case SC_STORAGE_F16_SCALED: occupancy_aa<StF16S>(&po, &co); break;
    case SC_STORAGE_BF16: occupancy_aa<StBF16>(&po, &co); break;
    default: occupancy_aa<StF32>(&po, &co);
  }
  if (po < 1 || co < 1)
    return fail(SC_ECUDA, "the in-place step kernels cannot be made resident: %s", cudaGetErrorString(cudaGetLastError()));
  const long long units = h->lay.aa_units;
  h->grid = (int)std::max(1LL, std::min({(long long)sms * co, h->lay.nslots, units}));
  h->grid_psi = (int)std::max(1LL, std::min((long long)sms * po, units));
  h->zmax = 1;
  h->lay.tx = kAAThreads;
  h->lay.ty = 1;
  h->persist = false;
  h->wait_limit_ns = 2000000000LL;
  h->withhold = -1;
  // the persistent step wins where each of its CTAs has a large tile per plane (measured
  // at 512^3: 12.0k against 10.7k MLUPS); on small planes (128^3: 3.8k against 10.6k)
  // the two-pass step is the automatic choice
  const bool large_planes = (long long)h->p.nx * h->p.ny >= (1LL << 17);
  if (h->p.staging == SC_STAGING_PERSISTENT || (h->p.staging == SC_STAGING_AUTO && large_planes)) {
    h->persist = plan_persist(h);
    if (!h->persist && h->p.staging == SC_STAGING_PERSISTENT)
      return fail(SC_EINVAL, "the persistent in-place step is not available here: %s", h->persist_why);
    if (h->persist) apply_persist(h);
  }
  return SC_OK;
}

template <class S>
void* persist_fn(int nt) { return nt == 128 ? (void*)k_aa_persist<S, 128> : (void*)k_aa_persist<S, 256>; }

void* persist_kernel(int storage, int nt) {
  switch (storage) {
    case SC_STORAGE_F16: return persist_fn<StF16>(nt);
    case SC_STORAGE_F16_SCALED: return persist_fn<StF16S>(nt);
    case SC_STORAGE_BF16: return persist_fn<StBF16>(nt);
    default: return persist_fn<StF32>(nt);
  }
}

// Tile grid of the persistent in-place step over a band: cx x cy tile columns, one
// resident CTA each (a cooperative launch), chosen to minimise the busiest SM's work
// per plane in warp rounds (its CTAs' collisions plus the Psi of their tiles and
// halos, about a third of a collision per cell), counting a single CTA per SM (8
// warps) as three quarters as efficient as two. Tiles narrower than 2 sites (the ragged last tile included) are allowed only
// when one tile spans the axis, so that every slot a CTA reads for its halo belongs
// to a direct neighbour. Returns false when no grid fits (the two-pass step is used
// then).
// Steps per persistent launch: at most kPersistMaxSteps, and few enough that the
// launch's counters (K B (nz + 2) values) stay below 2^32.
int persist_max_steps(const sc_lbm* h) {
  const long long per_step = (long long)h->pband * (h->p.nz + 2);
  return (int)std::max(1LL, std::min<long long>(kPersistMaxSteps, 4294967294LL / per_step));
}

bool plan_persist_bands(sc_lbm* h, int B);

// The persistent step's plan: the requested band count, or the fewest bands (powers
// of two dividing nx into bands of at least 2 sites) for which a tile grid fits.
// More bands keep a band's plane in the L2 between its two reads (at 512^3 FP32 one
// band reads 1.88x the algorithmic bytes from DRAM), but at 512^3 their smaller tiles
// and extra plane handshakes cost more than that saves (1 / 2 / 4 bands: 11.8k /
// 10.9k / 8.2k MLUPS); bands make the step possible where one band's tiles would not
// fit the shared ring (planes of 2^20 sites).
bool plan_persist(sc_lbm* h) {
  if (h->pband_req > 0) return plan_persist_bands(h, h->pband_req);
  for (int B = 1; B <= h->p.nx / 2 || B == 1; B *= 2) {
    if (h->p.nx % B != 0) break;
    if (plan_persist_bands(h, B)) return true;
  }
  return false;
}

bool plan_persist_bands(sc_lbm* h, int B) {
  const sc_params* p = &h->p;
  const int bw = p->nx / B;  // the band width: tiles cover [b bw, (b + 1) bw)
  int dev = 0, sms = 1, coop = 0, smem_optin = 0;
  h->persist_why = "the device query failed";
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
  h->persist_why = "the device has no cooperative launch";
  if (!coop) return false;
  const long long cap = std::min<long long>(kMaxCtas, h->lay.nslots);
  double best = 1e300;
  bool found = false;
  // threads per CTA: sc_params.tile 1 = 128; otherwise 256 (measured faster at 256^3 and
  // 512^3)
  for (int nt : {128, 256}) {
    if ((p->tile == 1) != (nt == 128)) continue;
    void* fn = persist_kernel(p->storage, nt);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    // dynamic shared memory up to the opt-in limit less the kernel's static shared memory
    const int dyn_max = smem_optin - (int)fa.sharedSizeBytes;
    if (dyn_max <= 0 || cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_max) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    for (int cx = 1; cx <= bw && cx <= cap; ++cx) {
      const int tx = (bw + cx - 1) / cx, cxr = (bw + tx - 1) / tx;
      if (cxr != cx) continue;  // the same tiles as a smaller cx
      // a halo site's arrived populations lie up to two sites from the tile: every tile,
      // the ragged last one included, must be at least 2 wide so they belong to a direct
      // neighbour (or to the tile itself)
      if (cxr > 1 && bw - (cxr - 1) * tx < 2) continue;
      for (int cy = 1; cy <= p->ny && (long long)cx * cy <= cap; ++cy) {
        const int ty = (p->ny + cy - 1) / cy, cyr = (p->ny + ty - 1) / ty;
        if (cyr != cy) continue;
        if (cyr > 1 && p->ny - (cyr - 1) * ty < 2) continue;
        const size_t smem = (size_t)kRingSlots * (tx + 2) * (ty + 2) * sizeof(float2);
        if (smem > (size_t)dyn_max) continue;
        int occ = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, nt, smem) != cudaSuccess) {
          cudaGetLastError();
          continue;
        }
        const long long C = (long long)cx * cy;
        if (occ < 1 || C > (long long)occ * sms) continue;
        // warp rounds per plane on the busiest SM (collisions, plus the Psi of tile and
        // halo at about a third of a collision): the CTAs of an SM share its issue slots,
        // so a partly filled round costs its warps, not the whole CTA; an SM with fewer
        // than 16 resident warps counts as three quarters as efficient
        const long long per_sm = (C + sms - 1) / sms;
        const double rounds = std::ceil((double)tx * ty / 32) + 0.35 * std::ceil((double)(tx + 2) * (ty + 2) / 32);
        const double cost = (double)per_sm * rounds / (per_sm * nt >= 512 ? 1.0 : 0.75);
        if (cost < best * (1.0 - 1e-9)) {
          best = cost;
          found = true;
          h->pcx = cx; h->pcy = cy; h->ptx = tx; h->pty = ty; h->psmem = smem; h->pnt = nt; h->pband = B;
        }
      }
    }
  }
  h->persist_why = found ? "" : "no tile grid keeps one CTA per tile column resident";
  return found;
}

template <class S>
cudaError_t launch_persist_t(sc_lbm* h, int K, cudaStream_t st) {
  AAPersist a{};
  a.cx = h->pcx; a.cy = h->pcy; a.TX = h->ptx; a.TY = h->pty;
  a.B = h->pband;
  a.bw = h->p.nx / h->pband;
  a.edge = h->psi();  // the two-pass step's Psi array (np >= B nz ny entries), unused here
  a.K = K;
  a.odd0 = h->cur;
  a.epoch = (unsigned long long)(++h->launch_no) << 32;
  a.psi_done = h->flags();
  a.steps_done = h->flags() + kMaxCtas;
  a.err = h->err();
  a.limit_ns = h->wait_limit_ns;
  a.withhold = h->withhold;
  LatDev L = h->L;
  typename S::T* A = (typename S::T*)h->pop(0);
  double* evap = h->evap();
  void* args[] = {&L, &A, &evap, &a};
  return cudaLaunchCooperativeKernel(persist_fn<S>(h->pnt), dim3((unsigned)(h->pcx * h->pcy)), dim3(h->pnt), args,
                                     h->psmem, st);
}

// K in-place steps in one cooperative launch.
int launch_persist(sc_lbm* h, int K, cudaStream_t st) {
  cudaError_t e;
  switch (h->p.storage) {
    case SC_STORAGE_F16: e = launch_persist_t<StF16>(h, K, st); break;
    case SC_STORAGE_F16_SCALED: e = launch_persist_t<StF16S>(h, K, st); break;
    case SC_STORAGE_BF16: e = launch_persist_t<StBF16>(h, K, st); break;
    default: e = launch_persist_t<StF32>(h, K, st);
  }
  if (e != cudaSuccess) return fail(SC_ECUDA, "persistent in-place step launch failed: %s", cudaGetErrorString(e));
  if (K & 1) h->cur = 1 - h->cur;
  return SC_OK;
}

// The error word of the persistent step: SC_ETIMEOUT when one of its waits gave up
// (the lattice's state is then undefined until it is loaded again).
int persist_status(sc_lbm* h) {
  if (!h->persist) return SC_OK;
  int v = 0;
  CK(cudaMemcpyAsync(&v, h->err(), sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (v != 0)
    return fail(SC_ETIMEOUT, "a wait of the persistent in-place step gave up (%s); load a state to continue",
                v == 1 ? "between steps" : "between planes");
  return SC_OK;
}

int launch_one(sc_lbm* h, cudaStream_t st) {
  if (h->lay.aa) {
    cudaError_t e;
    switch (h->p.storage) {
      case SC_STORAGE_F16: e = launch_aa<StF16>(h, st); break;
      case SC_STORAGE_F16_SCALED: e = launch_aa<StF16S>(h, st); break;
      case SC_STORAGE_BF16: e = launch_aa<StBF16>(h, st); break;
      default: e = launch_aa<StF32>(h, st);
    }
    if (e != cudaSuccess) return fail(SC_ECUDA, "in-place step launch failed: %s", cudaGetErrorString(e));
    h->cur = 1 - h->cur;  // the lattice's form
    return SC_OK;
  }
  const int src = h->cur, dst = 1 - h->cur;
  StepArgs a{h->L, h->pop(src), h->pop(dst), h->evap(), h->lay.cols_x, h->items(), h->starts(), h->grid, st};
  cudaError_t e = step_ops(h->p.storage, h->lay.tile, h->lay.rows).launch(a);
  if (e != cudaSuccess) return fail(SC_ECUDA, "step launch failed: %s", cudaGetErrorString(e));
  h->cur = dst;
  return SC_OK;
}

unsigned grid_for(long long n, int threads) {
  return (unsigned)std::max(1LL, std::min<long long>((n + threads - 1) / threads, 152LL * 16));
}

template <class S>
int launch_canonical(sc_lbm* h, long long s0, long long s1, float* rho, long long rs, float* f, long long fs) {
  k_canonical<S><<<grid_for(s1 - s0, 256), 256, 0, h->stream>>>(h->L, (const typename S::T*)h->pop(h->cur), s0, s1,
                                                                  rho, rs, f, fs, h->odd());
  CK(cudaGetLastError());
  return SC_OK;
}

int canonical(sc_lbm* h, long long s0, long long s1, float* rho, long long rs, float* f, long long fs) {
  switch (h->p.storage) {
    case SC_STORAGE_F16: return launch_canonical<StF16>(h, s0, s1, rho, rs, f, fs);
    case SC_STORAGE_F16_SCALED: return launch_canonical<StF16S>(h, s0, s1, rho, rs, f, fs);
    case SC_STORAGE_BF16: return launch_canonical<StBF16>(h, s0, s1, rho, rs, f, fs);
    default: return launch_canonical<StF32>(h, s0, s1, rho, rs, f, fs);
  }
}

template <class S>
int launch_load(sc_lbm* h, long long s0, long long s1, int mode, const float* f, long long fs, const float* rho,
                long long rs, const ShapeDev& sh) {
  // the pull reads the current buffer, so the load writes it
  k_load<S><<<grid_for(s1 - s0, 256), 256, 0, h->stream>>>(h->L, (typename S::T*)h->pop(h->cur), s0, s1, mode, f, fs,
                                                            rho, rs, sh, (long long)h->p.nx * h->p.ny * h->L.nzg);
  CK(cudaGetLastError());
  return SC_OK;
}

int load(sc_lbm* h, long long s0, long long s1, int mode, const float* f, long long fs, const float* rho,
         long long rs, const ShapeDev& sh) {
  // every caller loads the whole lattice; in place it is written in the even form
  // (the two-lattice pull's slots); a new state clears the persistent step's error
  if (h->lay.aa) h->cur = 0;
  if (h->persist) CK(cudaMemsetAsync(h->err(), 0, sizeof(int), h->stream));
  switch (h->p.storage) {
    case SC_STORAGE_F16: return launch_load<StF16>(h, s0, s1, mode, f, fs, rho, rs, sh);
    case SC_STORAGE_F16_SCALED: return launch_load<StF16S>(h, s0, s1, mode, f, fs, rho, rs, sh);
    case SC_STORAGE_BF16: return launch_load<StBF16>(h, s0, s1, mode, f, fs, rho, rs, sh);
    default: return launch_load<StF32>(h, s0, s1, mode, f, fs, rho, rs, sh);
  }
}

template <class S>
int launch_diag(sc_lbm* h) {
  dim3 grid(h->p.nz, h->lay.diag_nsplit);
  k_diag<S><<<grid, kDiagThreads, 0, h->stream>>>(h->L, (const typename S::T*)h->pop(h->cur), h->lay.diag_nsplit,
                                                  h->diag(), h->odd());
  CK(cudaGetLastError());
  return SC_OK;
}

// Whether local plane z lies in the solid slab (the whole lattice's plane numbers).
bool host_solid(const sc_lbm* h, int z) {
  int g = (z + h->L.zoff) % h->L.nzg;
  return h->L.wall_z0 <= g && g < h->L.wall_z1;
}

int reset_counters(sc_lbm* h) {
  CK(cudaMemsetAsync(h->evap(), 0, sizeof(double) * h->lay.nslots, h->stream));
  h->step = 0;
  h->evap_offset = 0.0;
  return SC_OK;
}

// Sites per slab so a slab's 2*19 FP32 populations fit the staging area.
long long slab_sites(const sc_lbm* h) { return std::max<long long>(1, (2 * h->lay.stage_n) / (2 * Q)); }

}  // namespace

namespace {
// Identity of the calling thread's current CUDA context (0 if the driver cannot
// say), through driver entry points that the runtime hands out, so the library
// needs no link against the driver library. A context destroyed by
// cudaDeviceReset and recreated gets a new identity.
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

unsigned long long current_context_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = (CtxGetCurrentFn)fn;
    fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)fn;
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

std::mutex g_noalloc_mu;
struct NoallocAddr {
  unsigned long long ctx;  // context the address belongs to (0: not looked up)
  double* ptr;
};
NoallocAddr g_noalloc_addr[128] = {};  // per device ordinal

// Device address of the file-scope scratch for the current device (host code may
// not use the symbol itself as a device pointer). It is looked up on the first
// call on a device and again whenever the device's context has changed since
// (after cudaDeviceReset the module, and with it the array, is loaded anew);
// when no context is current yet, or its identity is unavailable, it is looked
// up on every call (the lookup itself makes the primary context current).
int noalloc_scratch(double** out) {
  int dev = 0;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) return fail(SC_EINVAL, "device ordinal %d out of range", dev);
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  NoallocAddr& a = g_noalloc_addr[dev];
  if (ctx == 0 || a.ctx != ctx || !a.ptr) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    a.ptr = (double*)p;
    a.ctx = ctx;
  }
  *out = a.ptr;
  return SC_OK;
}

template <class S>
int launch_flux(sc_lbm* h) {
  dim3 grid(h->p.nz, h->lay.diag_nsplit);
  k_flux<S><<<grid, kDiagThreads, 0, h->stream>>>(h->L, (const typename S::T*)h->pop(h->cur), h->lay.diag_nsplit,
                                                  h->diag(), h->odd(), h->p.G, h->p.G_rr, h->p.G_bb);
  CK(cudaGetLastError());
  return SC_OK;
}

template <class S>
int launch_diag_into(sc_lbm* h, double* part) {
  dim3 grid(h->p.nz, h->lay.diag_nsplit);
  k_diag<S><<<grid, kDiagThreads, 0, h->stream>>>(h->L, (const typename S::T*)h->pop(h->cur), h->lay.diag_nsplit,
                                                  part, h->odd());
  CK(cudaGetLastError());
  return SC_OK;
}
}  // namespace

extern "C" {

const char* sc_last_error(void) { return g_err; }

int sc_lattice_directions(int32_t* c, double* w) {
  for (int i = 0; i < Q; ++i) {
    if (c) { c[3 * i] = dir_x(i); c[3 * i + 1] = dir_y(i); c[3 * i + 2] = dir_z(i); }
    if (w) w[i] = wgt_d(i);
  }
  return SC_OK;
}

int sc_tile_list(int32_t* count, int32_t* tx, int32_t* ty, int32_t capacity) {
  if (count) *count = kNumTiles;
  for (int k = 0; k < kNumTiles && k < capacity; ++k) {
    if (tx) tx[k] = kTileX[k];
    if (ty) ty[k] = kTileY[k];
  }
  return SC_OK;
}

int sc_lbm_required_bytes(const sc_params* p, size_t* bytes) {
  int rc = validate(p);
  if (rc) return rc;
  if (!bytes) return fail(SC_EINVAL, "bytes is NULL");
  *bytes = make_layout(p).total;
  return SC_OK;
}

static int create_common(const sc_params* p, void* stream, void* buf, bool owns, sc_lbm** out) {
  sc_lbm* h = new (std::nothrow) sc_lbm();
  if (!h) {
    if (owns) cudaFree(buf);
    return fail(SC_ENOMEM, "host allocation failed");
  }
  h->p = *p;
  h->lay = make_layout(p);
  h->L = make_dev(p, h->lay);
  h->stream = (cudaStream_t)stream;
  h->base = (char*)buf;
  h->owns = owns;
  h->cur = 0;
  int rc0 = SC_OK;
  if (h->lay.aa) {
    rc0 = plan_aa(h);
  } else {
    LaunchCfg cfg;
    rc0 = plan_launch(p, h->lay, h->lay.tile, p->zchunk, &cfg);
    if (!rc0) rc0 = apply_launch(h, cfg);
  }
  if (rc0) {
    sc_lbm_destroy(h);
    return rc0;
  }
  cudaError_t e = cudaMallocHost((void**)&h->h_diag, sizeof(double) * p->nz * h->lay.diag_nsplit * kDiagFields);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_evap, sizeof(double) * h->lay.nslots);
  if (e != cudaSuccess) {
    sc_lbm_destroy(h);
    return fail(SC_ENOMEM, "pinned host allocation failed: %s", cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(buf, 0, h->lay.off_stage, h->stream);
  if (e == cudaSuccess)
    e = cudaMemsetAsync((char*)buf + h->lay.off_flags, 0, h->lay.total - h->lay.off_flags, h->stream);
  if (e != cudaSuccess) {
    sc_lbm_destroy(h);
    return fail(SC_ECUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
  }
  int rc = reset_counters(h);
  if (rc) { sc_lbm_destroy(h); return rc; }
  *out = h;
  return SC_OK;
}

int sc_lbm_create(const sc_params* p, void* stream, sc_lbm** out) {
  int rc = validate(p);
  if (rc) return rc;
  if (!out) return fail(SC_EINVAL, "out is NULL");
  const Layout l = make_layout(p);
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, l.total);
  if (e != cudaSuccess) return fail(SC_ENOMEM, "cudaMalloc(%zu) failed: %s", l.total, cudaGetErrorString(e));
  return create_common(p, stream, buf, true, out);
}

int sc_lbm_create_ext(const sc_params* p, void* stream, void* buf, size_t bytes, sc_lbm** out) {
  int rc = validate(p);
  if (rc) return rc;
  if (!out || !buf) return fail(SC_EINVAL, "NULL argument");
  if (((uintptr_t)buf & 255) != 0) return fail(SC_EINVAL, "device buffer must be 256-byte aligned");
  const Layout l = make_layout(p);
  if (bytes < l.total) return fail(SC_ENOMEM, "device buffer has %zu bytes, needs %zu", bytes, l.total);
  return create_common(p, stream, buf, false, out);
}

void sc_lbm_destroy(sc_lbm* h) {
  if (!h || h->owner) return;  // a batch member goes with sc_batch_remove / sc_batch_destroy
  cudaStreamSynchronize(h->stream);
  if (h->graph) cudaGraphExecDestroy(h->graph);
  if (h->h_diag) cudaFreeHost(h->h_diag);
  if (h->h_evap) cudaFreeHost(h->h_evap);
  if (h->owns && h->base) cudaFree(h->base);
  delete h;
}

int sc_lbm_set_stream(sc_lbm* h, void* stream) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  h->stream = (cudaStream_t)stream;
  return SC_OK;
}

int sc_lbm_sync(sc_lbm* h) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  return persist_status(h);
}

int sc_lbm_init(sc_lbm* h, const sc_init* in) {
  Range range("sc_lbm_init");
  if (!h || !in) return fail(SC_EINVAL, "NULL argument");
  if (in->shape < 0 || in->shape > 1) return fail(SC_EINVAL, "unknown shape %d", in->shape);
  if (!std::isfinite(in->rho_hi) || !std::isfinite(in->rho_lo) || !std::isfinite(in->noise_amp))
    return fail(SC_EINVAL, "densities must be finite");
  ShapeDev sh{};
  sh.shape = in->shape; sh.film_z = in->film_z;
  sh.cx = in->cx; sh.cy = in->cy; sh.cz = in->cz; sh.R2 = in->radius * in->radius;
  sh.hi = in->rho_hi; sh.lo = in->rho_lo; sh.amp = in->noise_amp; sh.seed = in->seed;
  int rc = load(h, 0, h->lay.nsites, 2, nullptr, 0, nullptr, 0, sh);
  if (rc) return rc;
  return reset_counters(h);
}

int sc_lbm_init_fields(sc_lbm* h, const float* rr, const float* rb) {
  Range range("sc_lbm_init_fields");
  if (!h || !rr || !rb) return fail(SC_EINVAL, "NULL argument");
  const long long n = h->lay.nsites;
  float* st = h->stage();
  CK(cudaMemcpyAsync(st, rr, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemcpyAsync(st + h->lay.stage_n, rb, sizeof(float) * n, cudaMemcpyHostToDevice, h->stream));
  ShapeDev sh{};
  int rc = load(h, 0, n, 1, nullptr, 0, st, h->lay.stage_n, sh);
  if (!rc) rc = reset_counters(h);
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  return SC_OK;
}

static int ensure_graph(sc_lbm* h) {
  if (h->graph) return SC_OK;
  // enough launches per replay that launch overhead is amortised on small lattices
  const long long n = h->lay.nsites;
  int len = (int)std::min<long long>(64, std::max<long long>(2, (1LL << 21) / std::max<long long>(n, 1)));
  len += len & 1;
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const int saved = h->cur;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = SC_OK;
  if (e == cudaSuccess) {
    for (int k = 0; k < len && rc == SC_OK; ++k) rc = launch_one(h, cs);
    e = cudaStreamEndCapture(cs, &g);
  }
  h->cur = saved;
  cudaStreamDestroy(cs);
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return fail(SC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { h->graph = nullptr; return fail(SC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e)); }
  h->graph_len = len;
  h->graph_cur = saved;
  return SC_OK;
}

static void batch_touch(sc_batch* b);  // the member's buffer parity changed outside the batch

int sc_lbm_step(sc_lbm* h, int64_t nsteps) {
  Range range("sc_lbm_step");
  if (!h) return fail(SC_EINVAL, "NULL handle");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  if (h->owner && nsteps > 0) batch_touch(h->owner);
  int64_t left = nsteps;
  if (h->persist) {
    while (left > 0) {
      const int k = (int)std::min<int64_t>(left, persist_max_steps(h));
      int rc = launch_persist(h, k, h->stream);
      if (rc) return rc;
      left -= k;
    }
    h->step += nsteps;
    return SC_OK;
  }
  if (left >= 4) {
    int rc = ensure_graph(h);
    if (rc) return rc;
  }
  while (left > 0) {
    if (h->graph && left >= h->graph_len && h->cur == h->graph_cur) {
      CK(cudaGraphLaunch(h->graph, h->stream));
      left -= h->graph_len;  // graph_len is even: the buffer parity is unchanged
    } else {
      int rc = launch_one(h, h->stream);
      if (rc) return rc;
      left -= 1;
    }
  }
  h->step += nsteps;
  return SC_OK;
}

int sc_lbm_read_fields_device(sc_lbm* h, float* rr, float* rb) {
  if (!h || !rr || !rb) return fail(SC_EINVAL, "NULL argument");
  int rc = canonical(h, 0, h->lay.nsites, h->stage(), h->lay.stage_n, nullptr, 0);
  if (rc) return rc;
  CK(cudaMemcpyAsync(rr, h->stage(), sizeof(float) * h->lay.nsites, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(rb, h->stage() + h->lay.stage_n, sizeof(float) * h->lay.nsites, cudaMemcpyDeviceToDevice,
                     h->stream));
  return SC_OK;
}

int sc_lbm_read_fields(sc_lbm* h, float* rr, float* rb) {
  Range range("sc_lbm_read_fields");
  if (!h || !rr || !rb) return fail(SC_EINVAL, "NULL argument");
  int rc = canonical(h, 0, h->lay.nsites, h->stage(), h->lay.stage_n, nullptr, 0);
  if (rc) return rc;
  CK(cudaMemcpyAsync(rr, h->stage(), sizeof(float) * h->lay.nsites, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(rb, h->stage() + h->lay.stage_n, sizeof(float) * h->lay.nsites, cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SC_OK;
}

int sc_lbm_read_populations(sc_lbm* h, double* f) {
  Range range("sc_lbm_read_populations");
  if (!h || !f) return fail(SC_EINVAL, "NULL argument");
  const long long n = h->lay.nsites, slab = slab_sites(h);
  std::vector<float> tmp;
  try { tmp.resize((size_t)2 * Q * slab); } catch (...) { return fail(SC_ENOMEM, "host allocation failed"); }
  for (long long s0 = 0; s0 < n; s0 += slab) {
    const long long s1 = std::min(n, s0 + slab), m = s1 - s0;
    int rc = canonical(h, s0, s1, nullptr, 0, h->stage(), m);
    if (rc) return rc;
    CK(cudaMemcpyAsync(tmp.data(), h->stage(), sizeof(float) * 2 * Q * m, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int k = 0; k < 2 * Q; ++k)
      for (long long o = 0; o < m; ++o) f[(long long)k * n + s0 + o] = (double)tmp[(size_t)k * m + o];
  }
  return SC_OK;
}

int sc_lbm_write_populations(sc_lbm* h, const double* f) {
  Range range("sc_lbm_write_populations");
  if (!h || !f) return fail(SC_EINVAL, "NULL argument");
  const long long n = h->lay.nsites, slab = slab_sites(h);
  std::vector<float> tmp;
  try { tmp.resize((size_t)2 * Q * slab); } catch (...) { return fail(SC_ENOMEM, "host allocation failed"); }
  ShapeDev sh{};
  for (long long s0 = 0; s0 < n; s0 += slab) {
    const long long s1 = std::min(n, s0 + slab), m = s1 - s0;
    for (int k = 0; k < 2 * Q; ++k)
      for (long long o = 0; o < m; ++o) tmp[(size_t)k * m + o] = (float)f[(long long)k * n + s0 + o];
    CK(cudaMemcpyAsync(h->stage(), tmp.data(), sizeof(float) * 2 * Q * m, cudaMemcpyHostToDevice, h->stream));
    int rc = load(h, s0, s1, 0, h->stage(), m, nullptr, 0, sh);
    if (rc) return rc;
    CK(cudaStreamSynchronize(h->stream));  // tmp is reused for the next slab
  }
  return SC_OK;
}

int sc_lbm_set_counters(sc_lbm* h, int64_t step, double evaporated) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  CK(cudaMemsetAsync(h->evap(), 0, sizeof(double) * h->lay.nslots, h->stream));
  h->step = step;
  h->evap_offset = evaporated;
  return SC_OK;
}

static int run_diag(sc_lbm* h) {
  int rc;
  switch (h->p.storage) {
    case SC_STORAGE_F16: rc = launch_diag<StF16>(h); break;
    case SC_STORAGE_F16_SCALED: rc = launch_diag<StF16S>(h); break;
    case SC_STORAGE_BF16: rc = launch_diag<StBF16>(h); break;
    default: rc = launch_diag<StF32>(h);
  }
  if (rc) return rc;
  const size_t nd = (size_t)h->p.nz * h->lay.diag_nsplit * kDiagFields;
  CK(cudaMemcpyAsync(h->h_diag, h->diag(), sizeof(double) * nd, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemcpyAsync(h->h_evap, h->evap(), sizeof(double) * h->lay.nslots, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SC_OK;
}

int sc_lbm_flux_profile(sc_lbm* h, double* j) {
  Range range("sc_lbm_flux_profile");
  if (!h || !j) return fail(SC_EINVAL, "NULL argument");
  if (h->p.tau_r != 1.0 || h->p.tau_b != 1.0)
    return fail(SC_EINVAL, "the relative flux of Eqs. (flux) and (velw) is defined for tau = 1");
  int rc;
  switch (h->p.storage) {
    case SC_STORAGE_F16: rc = launch_flux<StF16>(h); break;
    case SC_STORAGE_F16_SCALED: rc = launch_flux<StF16S>(h); break;
    case SC_STORAGE_BF16: rc = launch_flux<StBF16>(h); break;
    default: rc = launch_flux<StF32>(h);
  }
  if (rc) return rc;
  const int nz = h->p.nz, ns = h->lay.diag_nsplit;
  const size_t nd = (size_t)nz * ns * kDiagFields;
  CK(cudaMemcpyAsync(h->h_diag, h->diag(), sizeof(double) * nd, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  const double nxy = (double)h->p.nx * h->p.ny;
  for (int d = 0; d < 3; ++d)
    for (int z = 0; z < nz; ++z) {
      double acc = 0.0;
      for (int k = 0; k < ns; ++k) acc += h->h_diag[((size_t)z * ns + k) * kDiagFields + d];
      j[(size_t)d * nz + z] = acc / nxy;
    }
  return SC_OK;
}

int sc_lbm_profile(sc_lbm* h, double* phi) {
  if (!h || !phi) return fail(SC_EINVAL, "NULL argument");
  int rc = run_diag(h);
  if (rc) return rc;
  const int ns = h->lay.diag_nsplit;
  const double nxy = (double)h->p.nx * h->p.ny;
  for (int z = 0; z < h->p.nz; ++z) {
    if (host_solid(h, z)) { phi[z] = NAN; continue; }
    double acc = 0.0;
    for (int k = 0; k < ns; ++k) acc += h->h_diag[((size_t)z * ns + k) * kDiagFields + 2];
    phi[z] = acc / nxy;
  }
  return SC_OK;
}

int sc_lbm_diagnostics(sc_lbm* h, sc_diag* d) {
  Range range("sc_lbm_diagnostics");
  if (!h || !d) return fail(SC_EINVAL, "NULL argument");
  int rc = run_diag(h);
  if (rc) return rc;
  std::memset(d, 0, sizeof(*d));
  const int nz = h->p.nz, ns = h->lay.diag_nsplit;
  const double nxy = (double)h->p.nx * h->p.ny;
  std::vector<double> phi(nz);
  double pending = 0.0, count = 0.0, nonfinite = 0.0, sinkneg = 0.0;
  for (int z = 0; z < nz; ++z) {
    double pz = 0.0;
    for (int k = 0; k < ns; ++k) {
      const double* q = h->h_diag + ((size_t)z * ns + k) * kDiagFields;
      d->mass_r += q[0];
      d->mass_b += q[1];
      pz += q[2];
      pending += q[3];
      count += q[4];
      nonfinite = std::max(nonfinite, q[5]);
      sinkneg = std::max(sinkneg, q[6]);
    }
    phi[z] = host_solid(h, z) ? NAN : pz / nxy;
  }
  double cum = 0.0;
  for (long long k = 0; k < h->lay.nslots; ++k) cum += h->h_evap[k];
  d->step = h->step;
  d->evaporated_mass = h->evap_offset + cum + pending;
  d->flux_last = pending;
  d->droplet_sites = (int64_t)count;
  d->radius = std::cbrt(3.0 * count / (4.0 * M_PI));
  const int z0 = h->L.wall_z1 > h->L.wall_z0 ? h->L.wall_z1 : 0;
  d->interface_z = -1.0;
  for (int z = z0; z + 1 < nz; ++z) {
    if (std::isnan(phi[z]) || std::isnan(phi[z + 1])) continue;
    if (phi[z] > 0.0 && phi[z + 1] <= 0.0) {
      d->interface_z = z + phi[z] / (phi[z] - phi[z + 1]);
      break;
    }
  }
  d->status = nonfinite > 0.0 ? SC_ENONFINITE : (sinkneg > 0.0 ? SC_ESINKNEG : SC_OK);
  if (!std::isfinite(d->mass_r) || !std::isfinite(d->mass_b)) d->status = SC_ENONFINITE;
  if (persist_status(h) == SC_ETIMEOUT) d->status = SC_ETIMEOUT;
  return SC_OK;
}

int sc_lbm_diagnostics_noalloc(sc_lbm* h, double* out_dev) {
  Range range("sc_lbm_diagnostics_noalloc");
  if (!h || !out_dev) return fail(SC_EINVAL, "NULL argument");
  if (h->slab) return fail(SC_EINVAL, "diagnostics without allocation take whole lattices, not slabs");
  const long long need = (long long)h->p.nz * h->lay.diag_nsplit * kDiagFields;
  if (need > kNoAllocScratch)
    return fail(SC_EINVAL, "diagnostics without allocation need %lld doubles of scratch, the limit is %lld (nz too large)",
                need, kNoAllocScratch);
  double* part = nullptr;
  int rc = noalloc_scratch(&part);
  if (rc) return rc;
  switch (h->p.storage) {
    case SC_STORAGE_F16: rc = launch_diag_into<StF16>(h, part); break;
    case SC_STORAGE_F16_SCALED: rc = launch_diag_into<StF16S>(h, part); break;
    case SC_STORAGE_BF16: rc = launch_diag_into<StBF16>(h, part); break;
    default: rc = launch_diag_into<StF32>(h, part);
  }
  if (rc) return rc;
  k_diag_finish<<<1, 1, 0, h->stream>>>(part, h->p.nz, h->lay.diag_nsplit, (double)h->p.nx * h->p.ny, h->L.wall_z0,
                                        h->L.wall_z1, h->evap(), h->lay.nslots, h->evap_offset,
                                        h->persist ? h->err() : nullptr, out_dev);
  CK(cudaGetLastError());
  return SC_OK;
}

int sc_lbm_launch_info(sc_lbm* h, int32_t* tx, int32_t* ty, int32_t* zchunk, int64_t* ctas, int32_t* staging) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  if (staging) *staging = h->persist ? SC_STAGING_PERSISTENT : (h->lay.rows ? SC_STAGING_ROWS : SC_STAGING_THREAD);
  if (tx) *tx = h->lay.tx;
  if (ty) *ty = h->lay.ty;
  if (zchunk) *zchunk = h->zmax;
  if (ctas) *ctas = h->grid;
  return SC_OK;
}

int sc_lbm_tune(sc_lbm* h, int32_t trials, int32_t* tile, int32_t* zchunk) {
  Range range("sc_lbm_tune");
  if (!h) return fail(SC_EINVAL, "NULL handle");
  if (h->lay.aa) {  // one configuration, and no spare buffer for trial launches
    if (tile) *tile = 0;
    if (zchunk) *zchunk = h->zmax;
    return SC_OK;
  }
  if (trials < 1) trials = 3;
  // trial launches book their evaporated mass in the read-out staging area and
  // use the handle's work-list buffer; the chosen list is uploaded at the end
  double* scratch = (double*)h->stage();
  const long long scratch_slots = h->lay.stage_n;  // 2 * stage_n floats
  LaunchCfg best;
  int rc = plan_launch(&h->p, h->lay, h->lay.tile, h->p.zchunk, &best);  // the current choice
  if (rc) return rc;
  float best_ms = 1e30f;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  static const int kZc[] = {0, 16, 32, 64};
  std::vector<LaunchCfg> tried;
  for (int t = 0; t < kNumTiles && rc == SC_OK; ++t)
    for (int zc : kZc) {
      LaunchCfg c;
      if (plan_launch(&h->p, h->lay, t, zc, &c) != SC_OK || c.grid > scratch_slots) continue;
      bool dup = false;
      for (const LaunchCfg& o : tried)
        dup = dup || (o.tile == c.tile && o.grid == c.grid && o.starts == c.starts && o.items.size() == c.items.size() &&
                      std::equal(o.items.begin(), o.items.end(), c.items.begin(), [](const int4& u, const int4& v) {
                        return u.x == v.x && u.y == v.y && u.z == v.z && u.w == v.w;
                      }));
      if (dup) continue;
      tried.push_back(c);
      cudaError_t e = cudaMemcpyAsync(h->items(), c.items.data(), sizeof(int4) * c.items.size(), cudaMemcpyHostToDevice,
                                      h->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->starts(), c.starts.data(), sizeof(int) * c.starts.size(), cudaMemcpyHostToDevice,
                            h->stream);
      StepArgs a{h->L, h->pop(h->cur), h->pop(1 - h->cur), scratch, c.cols_x, h->items(), h->starts(), c.grid, h->stream};
      const StepOps ops = step_ops(h->p.storage, t, h->lay.rows);
      if (e == cudaSuccess) e = ops.launch(a);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
      for (int k = 0; k < trials && e == cudaSuccess; ++k) e = ops.launch(a);
      if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { rc = fail(SC_ECUDA, "tuning trial failed: %s", cudaGetErrorString(e)); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best_ms) { best_ms = ms; best = c; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const int rc2 = apply_launch(h, best);  // also restores the work list after failed trials
  if (rc) return rc;
  if (rc2) return rc2;
  if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
  if (tile) *tile = h->lay.tile + 1;
  if (zchunk) *zchunk = h->zmax;
  return SC_OK;
}

// ------------------------------------------------------------------ z slabs of one lattice

int sc_slab_create(const sc_params* g, int32_t z0, int32_t z1, void* stream, sc_lbm** out) {
  int rc = validate(g);
  if (rc) return rc;
  if (!out) return fail(SC_EINVAL, "out is NULL");
  if (g->layout != SC_LAYOUT_TWO_LATTICE) return fail(SC_EINVAL, "slabs use the two-lattice layout");
  if (z0 < 0 || z1 > g->nz || z1 - z0 < kSlabGhosts)
    return fail(SC_EINVAL, "slab planes [%d, %d) must lie in [0, %d) and number at least %d", z0, z1, g->nz,
                kSlabGhosts);
  const int nloc = z1 - z0 + 2 * kSlabGhosts;
  if ((long long)g->nx * g->ny * nloc > (1LL << 31) - 4096) return fail(SC_EINVAL, "slab too large");
  // the handle's own parameters describe the local planes; the geometry stays the whole
  // lattice's (set in its LatDev below)
  sc_params lp = *g;
  lp.nz = nloc;
  lp.wall_thickness = 0;
  lp.wall_z0 = 0;
  lp.sink_z0 = 0;
  lp.sink_layers = std::min(g->sink_layers, nloc);
  if (lp.geometry == SC_GEOM_PLANAR_SINK && lp.sink_layers < 1) lp.sink_layers = 1;
  const Layout l = make_layout(&lp);
  void* buf = nullptr;
  cudaError_t e = cudaMalloc(&buf, l.total);
  if (e != cudaSuccess) return fail(SC_ENOMEM, "cudaMalloc(%zu) failed: %s", l.total, cudaGetErrorString(e));
  sc_lbm* h = nullptr;
  rc = create_common(&lp, stream, buf, true, &h);
  if (rc) return rc;
  const LatDev G = make_dev(g, l);
  h->L.wall_z0 = G.wall_z0;
  h->L.wall_z1 = G.wall_z1;
  h->L.sink_z0 = G.sink_z0;
  h->L.sink_layers = G.sink_layers;
  h->L.nzg = g->nz;
  h->L.zoff = ((z0 - kSlabGhosts) % g->nz + g->nz) % g->nz;
  h->L.own0 = kSlabGhosts;
  h->L.own1 = kSlabGhosts + (z1 - z0);
  h->slab = true;
  *out = h;
  return SC_OK;
}

int sc_slab_info(sc_lbm* h, int32_t* z0, int32_t* z1, int32_t* ghosts, size_t* face_bytes) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  if (!h->slab) return fail(SC_EINVAL, "not a slab");
  if (z0) *z0 = (h->L.zoff + kSlabGhosts) % h->L.nzg;
  if (z1) *z1 = (h->L.zoff + kSlabGhosts) % h->L.nzg + (h->L.own1 - h->L.own0);
  if (ghosts) *ghosts = kSlabGhosts;
  if (face_bytes) *face_bytes = (size_t)2 * Q * kSlabGhosts * h->p.nx * h->p.ny * elem_size(h->p.storage);
  return SC_OK;
}

// The kSlabGhosts planes starting at local plane zl of the current buffer, as 2 * 19
// arrays of kSlabGhosts * nx * ny elements each, to or from a packed device buffer.
static int slab_copy(sc_lbm* h, int zl, void* packed, bool to_packed) {
  const size_t es = elem_size(h->p.storage);
  const size_t run = (size_t)kSlabGhosts * h->p.nx * h->p.ny * es;  // contiguous in each array
  char* planes = (char*)h->pop(h->cur) + (size_t)zl * h->p.nx * h->p.ny * es;
  const size_t pitch = (size_t)h->lay.np * es;
  if (to_packed)
    CK(cudaMemcpy2DAsync(packed, run, planes, pitch, run, 2 * Q, cudaMemcpyDeviceToDevice, h->stream));
  else
    CK(cudaMemcpy2DAsync(planes, pitch, packed, run, run, 2 * Q, cudaMemcpyDeviceToDevice, h->stream));
  return SC_OK;
}

int sc_slab_pack(sc_lbm* h, int32_t side, void* out_dev) {
  if (!h || !out_dev) return fail(SC_EINVAL, "NULL argument");
  if (!h->slab) return fail(SC_EINVAL, "not a slab");
  if (side != 0 && side != 1) return fail(SC_EINVAL, "side must be 0 (low) or 1 (high)");
  return slab_copy(h, side == 0 ? h->L.own0 : h->L.own1 - kSlabGhosts, out_dev, true);
}

int sc_slab_unpack(sc_lbm* h, int32_t side, const void* in_dev) {
  if (!h || !in_dev) return fail(SC_EINVAL, "NULL argument");
  if (!h->slab) return fail(SC_EINVAL, "not a slab");
  if (side != 0 && side != 1) return fail(SC_EINVAL, "side must be 0 (low) or 1 (high)");
  return slab_copy(h, side == 0 ? 0 : h->L.own1, (void*)in_dev, false);
}

int sc_lbm_launch_count(sc_lbm* h, int64_t nsteps, int64_t* launches) {
  if (!h || !launches) return fail(SC_EINVAL, "NULL argument");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  if (h->persist) *launches = (nsteps + persist_max_steps(h) - 1) / persist_max_steps(h);
  else *launches = h->lay.aa ? 2 * nsteps : nsteps;
  return SC_OK;
}

const char* sc_lbm_kernel_name(sc_lbm* h) {
  if (!h) return "";
  if (h->persist) return "k_aa_persist (cooperative; up to 1024 steps per launch)";
  if (h->lay.aa) return "k_aa_psi + k_aa_collide";
  return h->lay.rows ? "k_step (staged rows)" : "k_step (per-thread pulls)";
}

int sc_lbm_set_wait(sc_lbm* h, int64_t limit_ns, int32_t withhold_cta) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  if (limit_ns <= 0) return fail(SC_EINVAL, "limit_ns must be > 0");
  if (withhold_cta < -1 || (h->persist && withhold_cta >= h->pcx * h->pcy))
    return fail(SC_EINVAL, "withhold_cta out of range");
  h->wait_limit_ns = limit_ns;
  h->withhold = withhold_cta;
  return SC_OK;
}

int sc_lbm_persist_bands(sc_lbm* h, int32_t request, int32_t* bands) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  if (request < -1) return fail(SC_EINVAL, "request must be -1, 0 or a band count");
  if (request >= 0) {
    if (!h->persist) return fail(SC_EINVAL, "the lattice does not use the persistent in-place step");
    if (request > 1 && (h->p.nx % request != 0 || h->p.nx / request < 2))
      return fail(SC_EINVAL, "%d bands must divide nx = %d into bands of at least 2 sites", request, h->p.nx);
    const int old = h->pband_req;
    h->pband_req = request;
    if (!plan_persist(h)) {
      const char* why = h->persist_why;
      h->pband_req = old;
      plan_persist(h);  // the previous plan, which fitted
      apply_persist(h);
      return fail(SC_EINVAL, "no persistent plan with %d bands: %s", request, why);
    }
    apply_persist(h);
  }
  if (bands) *bands = h->persist ? h->pband : 0;
  return SC_OK;
}

int sc_lbm_diag_bytes(sc_lbm* h, size_t* bytes) {
  if (!h || !bytes) return fail(SC_EINVAL, "NULL argument");
  *bytes = sizeof(double) * ((size_t)h->p.nz * h->lay.diag_nsplit * kDiagFields + (size_t)h->lay.nslots);
  return SC_OK;
}

}  // extern "C"

#include "sc_batch.cuh"
#include "sc_ncomp.cuh"
