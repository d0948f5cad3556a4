// N-component step (2 to 4 components): the paper calls the extension of its
// two-component model to more components straightforward (Sec. I), and the force of
// Eq. (3) already sums over the other components cbar. Included at the end of
// sc_lbm.cu, whose device functions it shares; include/sc_lbm.h documents the
// sc_ncomp_* contract.
//
// Periodic lattice with an optional solid slab (halfway bounce-back, Psi = 0 at
// solid sites); no evaporation sink (the paper states it for two components).
// Two population lattices of FP32 arrays f[c][i][s]; each step is one launch of
// k_n_step: a CTA of 32 x 8 threads owns a tile column and a chunk of its planes and
// marches them, forming Psi^c of plane p + 1 over the tile and a one-site halo from
// the pulled populations into a shared ring of 4 planes, then pulling plane p again
// (an L2 hit), forming every component's force from the ring, the common velocity
// and the shifted relaxation, and storing f*. The per-component arithmetic is the
// two-component kernels' (sum19, psi_of, momentum, force_sum_one = force_sums per
// component, relax_core), and the sums over components are ordered so that two
// components give their bits.

namespace {

constexpr int kMaxComp = 4;

struct NDev {
  LatDev L;  // extents, array stride, solid slab (no sinks)
  float om[kMaxComp], tau[kMaxComp];
  float g[kMaxComp][kMaxComp];
};

// Pulled populations of one component (the arrays of component c start at src_c).
__device__ __forceinline__ void pull_comp(const LatDev& L, const float* __restrict__ src_c, const PullIdx& P,
                                          float (&f)[Q]) {
  Unroll<0, Q>::run([&](auto ic) {
    constexpr int I = decltype(ic)::value;
    int idx, d;
    P.template at<I>(idx, d);
    f[I] = __ldg(src_c + (long long)d * L.np + idx);
  });
}

constexpr int kNTX = 32, kNTY = 8, kNT = kNTX * kNTY;  // tile of the N-component step
constexpr int kNRW = kNTX + 2, kNRH = kNTY + 2;         // with its one-site halo

// Psi^c of 4 rolling planes (slot q & 3) over a tile and its halo.
template <int NC>
struct NRing {
  float v[4][NC][kNRH][kNRW];
};

// Psi of every component of plane q (any integer; periodic) over the tile at (x0, y0)
// and its halo into ring slot q & 3.
template <int NC>
__device__ __forceinline__ void n_psi_plane(const NDev& D, const float* __restrict__ src, NRing<NC>& r, int q,
                                            int x0, int y0) {
  const LatDev& L = D.L;
  const int zq = wrapi(q, L.nz), sl = q & 3;
  const bool solid = solid_z(L, zq);
  for (int h = threadIdx.x; h < kNRH * kNRW; h += kNT) {
    const int hx = h % kNRW, hy = h / kNRW;
    if (solid) {
#pragma unroll
      for (int c = 0; c < NC; ++c) r.v[sl][c][hy][hx] = 0.f;
      continue;
    }
    const int x = wrap_near(x0 + hx - 1, L.nx), y = wrap_near(y0 + hy - 1, L.ny);
    const PullIdx P(L, x, y, zq);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float f[Q];
      pull_comp(L, src + (long long)c * Q * L.np, P, f);
      r.v[sl][c][hy][hx] = psi_of(sum19(f));
    }
  }
}

// Stream, force, common velocity and shifted relaxation of site (x, y, p) (tile cell
// (tx, ty)), Psi from the ring; stores f*.
template <int NC>
__device__ __forceinline__ void n_collide_site(const NDev& D, const float* __restrict__ src, float* __restrict__ dst,
                                               const NRing<NC>& r, int p, int x, int y, int tx, int ty) {
  const LatDev& L = D.L;
  const PullIdx P(L, x, y, p);
  const int s = P.s;
  float f[NC][Q], rho[NC], m[NC][3];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    pull_comp(L, src + (long long)c * Q * L.np, P, f[c]);
    rho[c] = sum19(f[c]);
    momentum(f[c], m[c]);
  }
  // u' = sum_c m^c om_c / sum_c rho^c om_c, summed from the last component down (the
  // two-component kernels' order for NC = 2)
  float den = __fmul_rn(rho[NC - 1], D.om[NC - 1]);
#pragma unroll
  for (int c = NC - 2; c >= 0; --c) den = __fmaf_rn(rho[c], D.om[c], den);
  const float inv = den > 0.0f ? __fdiv_rn(1.0f, den) : 0.0f;
  float up[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    float num = __fmul_rn(m[NC - 1][d], D.om[NC - 1]);
#pragma unroll
    for (int c = NC - 2; c >= 0; --c) num = __fmaf_rn(m[c][d], D.om[c], num);
    up[d] = __fmul_rn(num, inv);
  }
  // a^c = sum_i w_i Psi^c(x + e_i) e_i from the ring (planes p - 1, p, p + 1)
  float a[NC][3];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    auto psi1 = [&](int sl, int yy, int xx) { return r.v[sl][c][yy + 1][xx + 1]; };
    force_sum_one(psi1, (p - 1) & 3, p & 3, (p + 1) & 3, ty, tx, a[c]);
  }
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    // A^c = sum_cbar g^{c cbar} a^cbar: the other components first (the first as a
    // product, the rest as fused multiply-adds), the self coupling last
    float A[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      float acc = 0.0f;
      bool first = true;
#pragma unroll
      for (int cb = 0; cb < NC; ++cb) {
        if (cb == c) continue;
        acc = first ? __fmul_rn(D.g[c][cb], a[cb][d]) : __fmaf_rn(D.g[c][cb], a[cb][d], acc);
        first = false;
      }
      A[d] = __fmaf_rn(D.g[c][c], a[c][d], acc);
    }
    relax_core(D.om[c], D.tau[c], f[c], rho[c], r.v[p & 3][c][ty + 1][tx + 1], 1.0f, A, up);
#pragma unroll
    for (int i = 0; i < Q; ++i) dst[((long long)c * Q + i) * L.np + s] = f[c][i];
  }
}

// One step: CTA (column, chunk) marches planes [zb, ze) of its tile column, one
// barrier per plane. Psi of plane p + 2 goes to ring slot (p + 2) & 3 while other
// threads may still collide plane p (slots p - 1, p, p + 1); the barrier after it
// is passed only when every thread has collided plane p.
template <int NC>
__global__ void __launch_bounds__(kNT) k_n_step(const NDev D, const float* __restrict__ src, float* __restrict__ dst,
                                                int cols_x, int cols, int nch) {
  __shared__ NRing<NC> r;
  const LatDev& L = D.L;
  const int col = (int)blockIdx.x % cols, k = (int)blockIdx.x / cols;
  const int x0 = (col % cols_x) * kNTX, y0 = (col / cols_x) * kNTY;
  const int zb = (int)((long long)k * L.nz / nch), ze = (int)((long long)(k + 1) * L.nz / nch);
  const int tx = (int)threadIdx.x % kNTX, ty = (int)threadIdx.x / kNTX;
  const int x = x0 + tx, y = y0 + ty;
  const bool active = x < L.nx && y < L.ny;
  n_psi_plane<NC>(D, src, r, zb - 1, x0, y0);
  n_psi_plane<NC>(D, src, r, zb, x0, y0);
  for (int p = zb; p < ze; ++p) {
    n_psi_plane<NC>(D, src, r, p + 1, x0, y0);
    __syncthreads();
    if (active && !solid_z(L, p)) n_collide_site<NC>(D, src, dst, r, p, x, y, tx, ty);
  }
}

// Canonical populations (pull) of every component into out[c][i][s] (dense, N sites).
template <int NC>
__global__ void k_n_canonical(const NDev D, const float* __restrict__ src, float* __restrict__ out) {
  const LatDev& L = D.L;
  const long long n = (long long)L.nxny * L.nz;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    site_of(L, s, x, y, z);
    const bool solid = site_class(L, x, y, z) == SOLID;
    const PullIdx P(L, x, y, z);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float f[Q];
      if (solid) {
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = 0.f;
      } else {
        pull_comp(L, src + (long long)c * Q * L.np, P, f);
      }
#pragma unroll
      for (int i = 0; i < Q; ++i) out[((long long)c * Q + i) * n + s] = f[i];
    }
  }
}

// Canonical populations in[c][i][s] (dense) written where the next pull reads them.
template <int NC>
__global__ void k_n_load(const NDev D, const float* __restrict__ in, float* __restrict__ dst) {
  const LatDev& L = D.L;
  const long long n = (long long)L.nxny * L.nz;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    site_of(L, s, x, y, z);
    if (site_class(L, x, y, z) == SOLID) continue;
#pragma unroll
    for (int c = 0; c < NC; ++c)
      Unroll<0, Q>::run([&](auto ic) {
        constexpr int I = decltype(ic)::value;
        const int zs = wrapi(z - dir_z(I), L.nz);
        const bool sol = dir_z(I) != 0 && solid_z(L, zs);
        const int idx = sol ? x + L.nx * y + L.nxny * z
                            : wrapi(x - dir_x(I), L.nx) + L.nx * wrapi(y - dir_y(I), L.ny) + L.nxny * zs;
        const int d = sol ? opp(I) : I;
        dst[((long long)c * Q + d) * L.np + idx] = in[((long long)c * Q + I) * n + s];
      });
  }
}

// Rest populations w_i rho^c (Eq. 2 at u = 0) of densities rho[c][s] (dense) into
// out[c][i][s] (dense), the canonical form k_n_load places.
template <int NC>
__global__ void k_n_rest(const NDev D, const float* __restrict__ rho, float* __restrict__ out) {
  const LatDev& L = D.L;
  const long long n = (long long)L.nxny * L.nz;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float r = rho[c * n + s];
#pragma unroll
      for (int i = 0; i < Q; ++i) out[((long long)c * Q + i) * n + s] = rest_pop(i, r);
    }
  }
}

// Site-parallel kernels (what: 2 canonical, 3 load, 4 rest populations) on `grid` CTAs.
template <int NC>
cudaError_t n_launch(int what, const NDev& D, const float* a, float* b, int grid, cudaStream_t st) {
  switch (what) {
    case 2: k_n_canonical<NC><<<grid, 256, 0, st>>>(D, a, b); break;
    case 4: k_n_rest<NC><<<grid, 256, 0, st>>>(D, a, b); break;
    default: k_n_load<NC><<<grid, 256, 0, st>>>(D, a, b); break;
  }
  return cudaGetLastError();
}

cudaError_t n_dispatch(int nc, int what, const NDev& D, const float* a, float* b, int grid, cudaStream_t st) {
  switch (nc) {
    case 2: return n_launch<2>(what, D, a, b, grid, st);
    case 3: return n_launch<3>(what, D, a, b, grid, st);
    default: return n_launch<4>(what, D, a, b, grid, st);
  }
}

template <int NC>
cudaError_t n_step_launch(const NDev& D, const float* src, float* dst, int cols_x, int cols, int nch,
                          cudaStream_t st) {
  k_n_step<NC><<<cols * nch, kNT, 0, st>>>(D, src, dst, cols_x, cols, nch);
  return cudaGetLastError();
}

cudaError_t n_step_dispatch(int nc, const NDev& D, const float* src, float* dst, int cols_x, int cols, int nch,
                            cudaStream_t st) {
  switch (nc) {
    case 2: return n_step_launch<2>(D, src, dst, cols_x, cols, nch, st);
    case 3: return n_step_launch<3>(D, src, dst, cols_x, cols, nch, st);
    default: return n_step_launch<4>(D, src, dst, cols_x, cols, nch, st);
  }
}

int n_step_occupancy(int nc) {
  int occ = 0;
  cudaError_t e = nc == 2 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_n_step<2>, kNT, 0)
                : nc == 3 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_n_step<3>, kNT, 0)
                          : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_n_step<4>, kNT, 0);
  if (e != cudaSuccess) cudaGetLastError();
  return e == cudaSuccess ? occ : 0;
}

}  // namespace

struct sc_ncomp {
  sc_nparams p;
  NDev D;
  cudaStream_t stream;
  char* base;
  size_t pop_bytes, off_pop[2], off_psi, total;
  int cur;
  int grid;                  // CTAs of the site-parallel kernels
  int cols_x, cols, nch;     // the step's tile columns and plane chunks (cols * nch CTAs)
  int64_t step;
  float* pop(int k) const { return (float*)(base + off_pop[k]); }
  float* psi() const { return (float*)(base + off_psi); }
};

extern "C" {

int sc_ncomp_create(const sc_nparams* p, void* stream, sc_ncomp** out) {
  if (!p || !out) return fail(SC_EINVAL, "NULL argument");
  if (p->ncomp < 2 || p->ncomp > kMaxComp) return fail(SC_EINVAL, "ncomp must be in [2, %d]", kMaxComp);
  if (p->nx < 1 || p->ny < 1 || p->nz < 1) return fail(SC_EINVAL, "lattice extents must be >= 1");
  if ((long long)p->nx * p->ny * p->nz > (1LL << 31) - 4096) return fail(SC_EINVAL, "lattice too large");
  for (int c = 0; c < p->ncomp; ++c) {
    if (!(p->tau[c] > 0.5) || !std::isfinite(p->tau[c])) return fail(SC_EINVAL, "tau must exceed 1/2");
    for (int b = 0; b < p->ncomp; ++b)
      if (!std::isfinite(p->g[c][b])) return fail(SC_EINVAL, "couplings must be finite");
  }
  if (p->wall_thickness < 0 || (p->wall_thickness > 0 && (p->wall_z0 < 0 || p->wall_z0 + p->wall_thickness > p->nz)))
    return fail(SC_EINVAL, "wall slab must lie inside [0, nz)");
  sc_ncomp* h = new (std::nothrow) sc_ncomp();
  if (!h) return fail(SC_ENOMEM, "host allocation failed");
  h->p = *p;
  sc_params q{};
  q.nx = p->nx; q.ny = p->ny; q.nz = p->nz;
  q.tau_r = q.tau_b = 1.0;
  q.wall_z0 = p->wall_z0; q.wall_thickness = p->wall_thickness;
  const Layout l = make_layout(&q);
  h->D.L = make_dev(&q, l);
  for (int c = 0; c < kMaxComp; ++c) {
    h->D.om[c] = c < p->ncomp ? (float)(1.0 / p->tau[c]) : 0.f;
    h->D.tau[c] = c < p->ncomp ? (float)p->tau[c] : 1.f;
    for (int b = 0; b < kMaxComp; ++b) h->D.g[c][b] = (c < p->ncomp && b < p->ncomp) ? (float)p->g[c][b] : 0.f;
  }
  const long long np = l.np;
  h->pop_bytes = align256((size_t)p->ncomp * Q * np * sizeof(float));
  h->off_pop[0] = 0;
  h->off_pop[1] = h->pop_bytes;
  h->off_psi = 2 * h->pop_bytes;
  h->total = h->off_psi + align256((size_t)p->ncomp * np * sizeof(float));
  h->stream = (cudaStream_t)stream;
  h->grid = (int)grid_for(l.nsites, 256);
  // plane chunks: the fewest waves of resident CTAs times the planes (with the two
  // halo planes) each CTA marches
  h->cols_x = (p->nx + kNTX - 1) / kNTX;
  h->cols = h->cols_x * ((p->ny + kNTY - 1) / kNTY);
  {
    int dev = 0, sms = 1;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long slots = (long long)std::max(1, sms) * std::max(1, n_step_occupancy(p->ncomp));
    double best = 1e300;
    h->nch = 1;
    for (int nch = 1; nch <= p->nz && (long long)nch * h->cols <= (1LL << 30); ++nch) {
      const long long waves = ((long long)h->cols * nch + slots - 1) / slots;
      const double cost = (double)waves * ((p->nz + nch - 1) / nch + 2);
      if (cost < best * (1.0 - 1e-9)) { best = cost; h->nch = nch; }
    }
  }
  cudaError_t e = cudaMalloc((void**)&h->base, h->total);
  if (e != cudaSuccess) {
    delete h;
    return fail(SC_ENOMEM, "cudaMalloc(%zu) failed: %s", h->total, cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(h->base, 0, h->total, h->stream);
  if (e != cudaSuccess) {
    cudaFree(h->base);
    delete h;
    return fail(SC_ECUDA, "cudaMemsetAsync failed: %s", cudaGetErrorString(e));
  }
  *out = h;
  return SC_OK;
}

void sc_ncomp_destroy(sc_ncomp* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->base);
  delete h;
}

int sc_ncomp_write_populations(sc_ncomp* h, const double* f) {
  Range range("sc_ncomp_write_populations");
  if (!h || !f) return fail(SC_EINVAL, "NULL argument");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz, m = (size_t)h->p.ncomp * Q * n;
  std::vector<float> tmp;
  try { tmp.resize(m); } catch (...) { return fail(SC_ENOMEM, "host allocation failed"); }
  for (size_t k = 0; k < m; ++k) tmp[k] = (float)f[k];
  // staged in the other buffer, which the next step overwrites anyway
  float* stage = h->pop(1 - h->cur);
  CK(cudaMemcpyAsync(stage, tmp.data(), sizeof(float) * m, cudaMemcpyHostToDevice, h->stream));
  CK(n_dispatch(h->p.ncomp, 3, h->D, stage, h->pop(h->cur), h->grid, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return SC_OK;
}

int sc_ncomp_init_fields(sc_ncomp* h, const float* rho) {
  Range range("sc_ncomp_init_fields");
  if (!h || !rho) return fail(SC_EINVAL, "NULL argument");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz;
  // densities into the Psi array (ncomp * np >= ncomp * n floats), their rest
  // populations into the other buffer, then placed where the next pull reads them
  float* stage = h->pop(1 - h->cur);
  CK(cudaMemcpyAsync(h->psi(), rho, sizeof(float) * h->p.ncomp * n, cudaMemcpyHostToDevice, h->stream));
  CK(n_dispatch(h->p.ncomp, 4, h->D, h->psi(), stage, h->grid, h->stream));
  CK(n_dispatch(h->p.ncomp, 3, h->D, stage, h->pop(h->cur), h->grid, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->step = 0;
  return SC_OK;
}

int sc_ncomp_read_populations(sc_ncomp* h, double* f) {
  Range range("sc_ncomp_read_populations");
  if (!h || !f) return fail(SC_EINVAL, "NULL argument");
  const size_t n = (size_t)h->p.nx * h->p.ny * h->p.nz, m = (size_t)h->p.ncomp * Q * n;
  std::vector<float> tmp;
  try { tmp.resize(m); } catch (...) { return fail(SC_ENOMEM, "host allocation failed"); }
  float* stage = h->pop(1 - h->cur);
  CK(n_dispatch(h->p.ncomp, 2, h->D, h->pop(h->cur), stage, h->grid, h->stream));
  CK(cudaMemcpyAsync(tmp.data(), stage, sizeof(float) * m, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (size_t k = 0; k < m; ++k) f[k] = (double)tmp[k];
  return SC_OK;
}

int sc_ncomp_step(sc_ncomp* h, int64_t nsteps) {
  Range range("sc_ncomp_step");
  if (!h) return fail(SC_EINVAL, "NULL handle");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  for (int64_t k = 0; k < nsteps; ++k) {
    const int src = h->cur, dst = 1 - h->cur;
    CK(n_step_dispatch(h->p.ncomp, h->D, h->pop(src), h->pop(dst), h->cols_x, h->cols, h->nch, h->stream));
    h->cur = dst;
  }
  h->step += nsteps;
  return SC_OK;
}

int sc_ncomp_sync(sc_ncomp* h) {
  if (!h) return fail(SC_EINVAL, "NULL handle");
  CK(cudaStreamSynchronize(h->stream));
  return SC_OK;
}

}  // extern "C"
