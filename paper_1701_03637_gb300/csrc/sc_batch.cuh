// Batched step: many lattices of different extents and parameters advanced by
// one persistent launch per time step (the method of Sec. II applied to each
// member unchanged). Included at the end of sc_lbm.cu, whose handle, layout and
// launch helpers it shares; include/sc_lbm.h documents the sc_batch_* contract.
//
// Work list: every member contributes its items (tile column, z chunk) in
// chunk-major order; members with longer items come first. CTAs claim items
// from a per-launch counter, so uneven lattices balance across the grid. A
// member's items carry its own LatDev, buffers and evaporated-mass slots (one
// slot per item, so the bookkeeping is deterministic whatever CTA runs it).
//
// A sequence of K launches (a CUDA graph for K = kBatchGraphLen) is followed by
// an advance kernel that moves each member's buffer parity and remaining-step
// count on the device; the host repeats the same arithmetic for its mirrors.
// Member m takes part in launch k of a sequence iff k < remaining_m, so every
// member stops exactly at its own step count.

namespace {

constexpr long long kUnlimited = INT64_MAX;  // remaining steps of a member without a limit

bool same_items(const std::vector<int2>& a, const std::vector<int2>& b) {
  if (a.size() != b.size()) return false;
  for (size_t i = 0; i < a.size(); ++i)
    if (a[i].x != b[i].x || a[i].y != b[i].y) return false;
  return true;
}

// One member lattice as the batched kernel sees it.
struct LatSlot {
  LatDev L;
  void* buf[2];         // the two population lattices
  double* evap;         // evaporated-mass slots, one per item
  long long remaining;  // steps left (launches this member still takes part in)
  int parity;           // buffer holding the member's pre-stream state
  int cols_x, cols, nch;
  int nslots;           // evaporated-mass slots of the member
};

template <int TX, int TY, class S>
__global__ void __launch_bounds__(TX * TY, (512 / (TX * TY)) > 1 ? 512 / (TX * TY) : 1)
    k_batch(const LatSlot* __restrict__ lats, const int2* __restrict__ items, int nitems,
            unsigned* __restrict__ next, int k, int trial) {
  using TileT = Tile<TX, TY, S>;
  using T = typename S::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  auto& sm = *reinterpret_cast<typename TileT::Smem*>(smem_raw);
  __shared__ LatSlot ls;
  __shared__ int s_it;
  TileT t(ls.L, sm, nullptr, nullptr);
  for (;;) {
    __syncthreads();  // the previous item's reads of the ring and of ls are over
    if (threadIdx.x == 0) s_it = (int)atomicAdd(next, 1u);
    __syncthreads();
    const int it = s_it;
    if (it >= nitems) break;
    const int2 w = items[it];
    {
      const int* from = reinterpret_cast<const int*>(lats + w.x);
      int* to = reinterpret_cast<int*>(&ls);
      for (int i = threadIdx.x; i < (int)(sizeof(LatSlot) / sizeof(int)); i += blockDim.x) to[i] = from[i];
    }
    __syncthreads();
    if ((long long)k >= ls.remaining) continue;
    const int par = (ls.parity + k) & 1;
    t.src = (const T*)ls.buf[par];
    t.dst = (T*)ls.buf[par ^ 1];
    t.evap = 0.0;
    const int kc = w.y / ls.cols, c = w.y - kc * ls.cols;
    const int zb = (int)((long long)kc * ls.L.nz / ls.nch), ze = (int)((long long)(kc + 1) * ls.L.nz / ls.nch);
    t.setup(c % ls.cols_x, c / ls.cols_x);
    t.run(zb, ze, (kc & 1) != 0);
    if (ls.L.geometry != 0) {
      const double e = t.block_evap();
      // a slot per item (batch_build checks that every member has a slot for each
      // of its items), so no two CTAs of a launch add to the same slot
      if (threadIdx.x == 0 && !trial) ls.evap[w.y] += e;
    }
  }
}

// End of a sequence of K launches: member m took min(K, remaining) steps.
__global__ void k_batch_advance(LatSlot* __restrict__ lats, int n, int K) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  const long long s = lats[m].remaining < K ? lats[m].remaining : K;
  lats[m].parity = (int)((lats[m].parity + s) & 1);
  if (lats[m].remaining != kUnlimited) lats[m].remaining -= s;
}

template <int TX, int TY, class S>
cudaError_t launch_batch(const LatSlot* lats, const int2* items, int nitems, unsigned* next, int k, int trial,
                         int grid, cudaStream_t st) {
  k_batch<TX, TY, S><<<grid, TX * TY, step_smem<TX, TY, S>(), st>>>(lats, items, nitems, next, k, trial);
  return cudaGetLastError();
}

template <int TX, int TY, class S>
int occupancy_batch() {
  int nb = 0;
  if (cudaFuncSetAttribute(k_batch<TX, TY, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)step_smem<TX, TY, S>()) != cudaSuccess)
    return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch<TX, TY, S>, TX * TY, step_smem<TX, TY, S>()) !=
      cudaSuccess)
    return 0;
  return nb;
}

using BatchLaunchFn = cudaError_t (*)(const LatSlot*, const int2*, int, unsigned*, int, int, int, cudaStream_t);
struct BatchOps {
  BatchLaunchFn launch;
  int (*occupancy)();
};

template <class S>
BatchOps pick_batch(int tile) {
  switch (tile) {
    case 0: return {&launch_batch<32, 8, S>, &occupancy_batch<32, 8, S>};
    case 1: return {&launch_batch<32, 4, S>, &occupancy_batch<32, 4, S>};
    case 2: return {&launch_batch<16, 8, S>, &occupancy_batch<16, 8, S>};
    case 4: return {&launch_batch<64, 4, S>, &occupancy_batch<64, 4, S>};
    default: return {&launch_batch<8, 4, S>, &occupancy_batch<8, 4, S>};
  }
}

BatchOps batch_ops(int storage, int tile) {
  switch (storage) {
    case SC_STORAGE_F16: return pick_batch<StF16>(tile);
    case SC_STORAGE_F16_SCALED: return pick_batch<StF16S>(tile);
    case SC_STORAGE_BF16: return pick_batch<StBF16>(tile);
    default: return pick_batch<StF32>(tile);
  }
}

constexpr int kBatchGraphLen = 32;  // launches per captured sequence
constexpr size_t kArenaAlign = 256;

// First-fit allocator over the batch's device arena (offsets, 256-byte aligned);
// freed ranges merge with their neighbours.
class Arena {
 public:
  void reset(size_t bytes) {
    free_.clear();
    if (bytes) free_.push_back({0, bytes});
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align256(bytes);
    for (size_t i = 0; i < free_.size(); ++i) {
      if (free_[i].size >= bytes) {
        *off = free_[i].off;
        free_[i].off += bytes;
        free_[i].size -= bytes;
        if (free_[i].size == 0) free_.erase(free_.begin() + (long)i);
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align256(bytes);
    size_t i = 0;
    while (i < free_.size() && free_[i].off < off) ++i;
    free_.insert(free_.begin() + (long)i, {off, bytes});
    if (i + 1 < free_.size() && free_[i].off + free_[i].size == free_[i + 1].off) {
      free_[i].size += free_[i + 1].size;
      free_.erase(free_.begin() + (long)i + 1);
    }
    if (i > 0 && free_[i - 1].off + free_[i - 1].size == free_[i].off) {
      free_[i - 1].size += free_[i].size;
      free_.erase(free_.begin() + (long)i);
    }
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (const auto& r : free_) s += r.size;
    return s;
  }
  size_t largest() const {
    size_t s = 0;
    for (const auto& r : free_) s = std::max(s, r.size);
    return s;
  }

 private:
  struct Range {
    size_t off, size;
  };
  std::vector<Range> free_;
};

}  // namespace

struct sc_batch {
  cudaStream_t stream;
  int storage;
  char* arena;
  size_t arena_bytes;
  Arena alloc;
  struct Member {
    sc_lbm* h;  // nullptr: free slot
    size_t off, bytes;
    long long remaining;
  };
  std::vector<Member> members;
  int tile;    // kernel tile (entry of the tile list)
  int zchunk;  // target planes per item
  // device work list (rebuilt when membership or configuration changes)
  bool dirty;
  LatSlot* d_lats;
  int2* d_items;
  unsigned* d_next;
  size_t cap_lats, cap_items;
  int nlat, nitems, grid;
  std::vector<int> order;  // member slot of each LatSlot entry
  cudaGraphExec_t graph;   // one sequence of kBatchGraphLen launches
  int graph_tile;
  std::vector<int2> graph_items;  // the work list the device holds
};

namespace {

void batch_drop_graph(sc_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
}

// Items of one member for the batch's tile and target chunk length: cols x nch,
// with nch near nz / zchunk and no more items than the member's evaporated-mass
// slots (a lattice has at least one slot per column of the smallest tile, so
// cols <= nslots for every tile and nch = 1 always fits).
int member_nch(const sc_lbm* h, int cols, int zchunk) {
  const long long nz = h->p.nz;
  long long nch = std::max(1LL, (nz + zchunk / 2) / std::max(1, zchunk));
  nch = std::min(nch, nz);
  nch = std::min(nch, std::max(1LL, h->lay.nslots / cols));
  return (int)nch;
}

int batch_build(sc_batch* b) {
  if (!b->dirty) return SC_OK;
  std::vector<int> slots;
  for (int m = 0; m < (int)b->members.size(); ++m)
    if (b->members[m].h) slots.push_back(m);
  // every member must use the batch's tile: re-plan its layout columns
  std::vector<LatSlot> lats;
  std::vector<double> cost;
  for (int m : slots) {
    sc_lbm* h = b->members[m].h;
    LatSlot s{};
    s.L = h->L;
    s.buf[0] = h->pop(0);
    s.buf[1] = h->pop(1);
    s.evap = h->evap();
    s.remaining = b->members[m].remaining;
    s.parity = h->cur;
    s.cols_x = (h->p.nx + kTileX[b->tile] - 1) / kTileX[b->tile];
    s.cols = s.cols_x * ((h->p.ny + kTileY[b->tile] - 1) / kTileY[b->tile]);
    s.nch = member_nch(h, s.cols, b->zchunk);
    s.nslots = (int)h->lay.nslots;
    if ((long long)s.cols * s.nch > h->lay.nslots)
      return fail(SC_EINVAL, "member %d has %lld items but %lld evaporated-mass slots", m,
                  (long long)s.cols * s.nch, h->lay.nslots);
    lats.push_back(s);
    cost.push_back((double)((h->p.nz + s.nch - 1) / s.nch + 2));
  }
  // longer items first (their lattice's items stay together, chunk-major)
  std::vector<int> idx(lats.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = (int)i;
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return cost[a] > cost[c]; });
  std::vector<LatSlot> sorted;
  b->order.clear();
  std::vector<int2> items;
  for (int i : idx) {
    const int j = (int)sorted.size();
    sorted.push_back(lats[i]);
    b->order.push_back(slots[i]);
    const int n = lats[i].cols * lats[i].nch;
    for (int w = 0; w < n; ++w) items.push_back(make_int2(j, w));
  }
  // a captured sequence stays valid while the work list keeps its shape and place
  const bool same_shape = b->graph && b->graph_tile == b->tile && b->nlat == (int)sorted.size() &&
                          b->nitems == (int)items.size() && sorted.size() <= b->cap_lats &&
                          items.size() <= b->cap_items && same_items(b->graph_items, items);
  if (!same_shape) batch_drop_graph(b);
  b->nlat = (int)sorted.size();
  b->nitems = (int)items.size();
  if (sorted.size() > b->cap_lats) {
    if (b->d_lats) cudaFree(b->d_lats);
    b->d_lats = nullptr;
    b->cap_lats = 0;
    CK(cudaMalloc((void**)&b->d_lats, sizeof(LatSlot) * sorted.size()));
    b->cap_lats = sorted.size();
  }
  if (items.size() > b->cap_items) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->cap_items = 0;
    CK(cudaMalloc((void**)&b->d_items, sizeof(int2) * items.size()));
    b->cap_items = items.size();
  }
  if (!sorted.empty()) {
    CK(cudaMemcpyAsync(b->d_lats, sorted.data(), sizeof(LatSlot) * sorted.size(), cudaMemcpyHostToDevice, b->stream));
    CK(cudaMemcpyAsync(b->d_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, b->stream));
    CK(cudaStreamSynchronize(b->stream));  // the host vectors go out of scope
  }
  const BatchOps ops = batch_ops(b->storage, b->tile);
  const int occ = ops.occupancy();
  int dev = 0, sms = 1;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (occ < 1) return fail(SC_ECUDA, "the batched kernel cannot be made resident");
  const int grid = (int)std::max(1LL, std::min<long long>((long long)occ * sms, b->nitems));
  if (grid != b->grid) batch_drop_graph(b);
  b->grid = grid;
  b->graph_items.swap(items);
  b->dirty = false;
  return SC_OK;
}

// K launches (trial: the state and the bookkeeping are left untouched) and, for
// a real sequence, the advance of every member.
int batch_sequence(sc_batch* b, cudaStream_t st, int K, bool trial) {
  if (b->nitems == 0) return SC_OK;
  const BatchOps ops = batch_ops(b->storage, b->tile);
  CK(cudaMemsetAsync(b->d_next, 0, sizeof(unsigned) * K, st));
  for (int k = 0; k < K; ++k) {
    cudaError_t e = ops.launch(b->d_lats, b->d_items, b->nitems, b->d_next + k, trial ? 0 : k, trial ? 1 : 0,
                               b->grid, st);
    if (e != cudaSuccess) return fail(SC_ECUDA, "batched step launch failed: %s", cudaGetErrorString(e));
  }
  if (!trial) {
    k_batch_advance<<<(b->nlat + 127) / 128, 128, 0, st>>>(b->d_lats, b->nlat, K);
    CK(cudaGetLastError());
  }
  return SC_OK;
}

// The host mirrors of a real sequence of K launches.
void batch_account(sc_batch* b, int K) {
  for (int j = 0; j < b->nlat; ++j) {
    sc_batch::Member& m = b->members[b->order[j]];
    const long long s = std::min<long long>(K, m.remaining);
    m.h->cur = (int)((m.h->cur + s) & 1);
    m.h->step += s;
    if (m.remaining != kUnlimited) m.remaining -= s;
  }
}

int batch_graph(sc_batch* b) {
  if (b->graph) return SC_OK;
  cudaStream_t cs;
  CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = SC_OK;
  if (e == cudaSuccess) {
    rc = batch_sequence(b, cs, kBatchGraphLen, false);
    e = cudaStreamEndCapture(cs, &g);
  }
  cudaStreamDestroy(cs);
  if (rc) { if (g) cudaGraphDestroy(g); return rc; }
  if (e != cudaSuccess) return fail(SC_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(&b->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) { b->graph = nullptr; return fail(SC_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e)); }
  b->graph_tile = b->tile;
  return SC_OK;
}

int batch_default_tile(const sc_batch* b) {
  int nx = 1 << 30, ny = 1 << 30;
  for (const auto& m : b->members)
    if (m.h) { nx = std::min(nx, m.h->p.nx); ny = std::min(ny, m.h->p.ny); }
  sc_params p{};
  p.nx = nx;
  p.ny = ny;
  return auto_tile(&p);
}

}  // namespace

static void batch_touch(sc_batch* b) { b->dirty = true; }

extern "C" {

int sc_batch_create(size_t arena_bytes, int32_t storage, void* stream, sc_batch** out) {
  if (!out) return fail(SC_EINVAL, "out is NULL");
  *out = nullptr;
  if (storage < 0 || storage > 3) return fail(SC_EINVAL, "unknown storage %d", storage);
  if (arena_bytes == 0) return fail(SC_EINVAL, "arena_bytes must be > 0");
  sc_batch* b = new (std::nothrow) sc_batch();
  if (!b) return fail(SC_ENOMEM, "host allocation failed");
  b->stream = (cudaStream_t)stream;
  b->storage = storage;
  b->tile = -1;
  b->zchunk = 32;
  b->dirty = true;
  cudaError_t e = cudaMalloc((void**)&b->arena, arena_bytes);
  if (e != cudaSuccess) {
    delete b;
    return fail(SC_ENOMEM, "cudaMalloc(%zu) failed: %s", arena_bytes, cudaGetErrorString(e));
  }
  b->arena_bytes = arena_bytes;
  b->alloc.reset(arena_bytes);
  e = cudaMalloc((void**)&b->d_next, sizeof(unsigned) * kBatchGraphLen);
  if (e != cudaSuccess) {
    cudaFree(b->arena);
    delete b;
    return fail(SC_ENOMEM, "cudaMalloc failed: %s", cudaGetErrorString(e));
  }
  *out = b;
  return SC_OK;
}

void sc_batch_destroy(sc_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  batch_drop_graph(b);
  for (auto& m : b->members)
    if (m.h) { m.h->owner = nullptr; sc_lbm_destroy(m.h); }
  if (b->d_lats) cudaFree(b->d_lats);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_next) cudaFree(b->d_next);
  if (b->arena) cudaFree(b->arena);
  delete b;
}

int sc_batch_add(sc_batch* b, const sc_params* p, int32_t* slot, sc_lbm** lattice) {
  if (!b || !p || !slot) return fail(SC_EINVAL, "NULL argument");
  int rc = validate(p);
  if (rc) return rc;
  if (p->storage != b->storage) return fail(SC_EINVAL, "the lattice's storage differs from the batch's");
  if (p->layout != SC_LAYOUT_TWO_LATTICE) return fail(SC_EINVAL, "batch members use the two-lattice layout");
  size_t bytes = 0;
  rc = sc_lbm_required_bytes(p, &bytes);
  if (rc) return rc;
  size_t off = 0;
  if (!b->alloc.alloc(bytes, &off))
    return fail(SC_ENOMEM, "batch arena full: %zu bytes needed, largest free range %zu", align256(bytes),
                b->alloc.largest());
  sc_lbm* h = nullptr;
  rc = sc_lbm_create_ext(p, b->stream, b->arena + off, bytes, &h);
  if (rc) {
    b->alloc.release(off, bytes);
    return rc;
  }
  h->owner = b;
  int s = 0;
  while (s < (int)b->members.size() && b->members[s].h) ++s;
  if (s == (int)b->members.size()) b->members.push_back({});
  b->members[s] = {h, off, bytes, kUnlimited};
  b->dirty = true;
  *slot = s;
  if (lattice) *lattice = h;
  return SC_OK;
}

int sc_batch_lattice(sc_batch* b, int32_t slot, sc_lbm** lattice) {
  if (!b || !lattice) return fail(SC_EINVAL, "NULL argument");
  if (slot < 0 || slot >= (int)b->members.size() || !b->members[slot].h) return fail(SC_EINVAL, "no member in slot %d", slot);
  *lattice = b->members[slot].h;
  return SC_OK;
}

int sc_batch_remove(sc_batch* b, int32_t slot) {
  if (!b) return fail(SC_EINVAL, "NULL batch");
  if (slot < 0 || slot >= (int)b->members.size() || !b->members[slot].h) return fail(SC_EINVAL, "no member in slot %d", slot);
  sc_batch::Member& m = b->members[slot];
  CK(cudaStreamSynchronize(b->stream));
  m.h->owner = nullptr;
  sc_lbm_destroy(m.h);
  b->alloc.release(m.off, m.bytes);
  m = {};
  b->dirty = true;
  return SC_OK;
}

int sc_batch_set_steps(sc_batch* b, int32_t slot, int64_t steps) {
  if (!b) return fail(SC_EINVAL, "NULL batch");
  if (slot < 0 || slot >= (int)b->members.size() || !b->members[slot].h) return fail(SC_EINVAL, "no member in slot %d", slot);
  b->members[slot].remaining = steps < 0 ? kUnlimited : steps;
  b->dirty = true;
  return SC_OK;
}

int sc_batch_remaining(sc_batch* b, int32_t slot, int64_t* steps) {
  if (!b || !steps) return fail(SC_EINVAL, "NULL argument");
  if (slot < 0 || slot >= (int)b->members.size() || !b->members[slot].h) return fail(SC_EINVAL, "no member in slot %d", slot);
  *steps = b->members[slot].remaining;
  return SC_OK;
}

int sc_batch_configure(sc_batch* b, int32_t tile, int32_t zchunk) {
  if (!b) return fail(SC_EINVAL, "NULL batch");
  if (tile < 0 || tile > kNumTiles) return fail(SC_EINVAL, "tile index out of range");
  if (zchunk < 0) return fail(SC_EINVAL, "zchunk must be >= 0");
  b->tile = tile > 0 ? tile - 1 : -1;
  b->zchunk = zchunk > 0 ? zchunk : 32;
  b->dirty = true;
  return SC_OK;
}

int sc_batch_step(sc_batch* b, int64_t nsteps) {
  Range range("sc_batch_step");
  if (!b) return fail(SC_EINVAL, "NULL batch");
  if (nsteps < 0) return fail(SC_EINVAL, "nsteps must be >= 0");
  if (b->tile < 0) { b->tile = batch_default_tile(b); b->dirty = true; }
  int rc = batch_build(b);
  if (rc) return rc;
  int64_t left = nsteps;
  while (left > 0) {
    if (left >= kBatchGraphLen) {
      rc = batch_graph(b);
      if (rc) return rc;
      CK(cudaGraphLaunch(b->graph, b->stream));
      batch_account(b, kBatchGraphLen);
      left -= kBatchGraphLen;
    } else {
      rc = batch_sequence(b, b->stream, (int)left, false);
      if (rc) return rc;
      batch_account(b, (int)left);
      left = 0;
    }
  }
  return SC_OK;
}

int sc_batch_tune(sc_batch* b, int32_t trials, int32_t* tile, int32_t* zchunk) {
  Range range("sc_batch_tune");
  if (!b) return fail(SC_EINVAL, "NULL batch");
  if (trials < 1) trials = 3;
  trials = std::min(trials, kBatchGraphLen);
  const int saved_tile = b->tile, saved_zc = b->zchunk;
  static const int kZc[] = {16, 32, 64};
  float best = 1e30f;
  int best_tile = saved_tile < 0 ? batch_default_tile(b) : saved_tile, best_zc = saved_zc;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = SC_OK;
  for (int t = 0; t < kNumTiles && rc == SC_OK; ++t)
    for (int zc : kZc) {
      b->tile = t;
      b->zchunk = zc;
      b->dirty = true;
      rc = batch_build(b);
      if (rc) break;
      rc = batch_sequence(b, b->stream, 1, true);  // warm-up
      if (rc) break;
      cudaEventRecord(e0, b->stream);
      rc = batch_sequence(b, b->stream, trials, true);
      if (rc) break;
      cudaEventRecord(e1, b->stream);
      cudaError_t e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) { rc = fail(SC_ECUDA, "tuning trial failed: %s", cudaGetErrorString(e)); break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; best_tile = t; best_zc = zc; }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->tile = rc ? saved_tile : best_tile;
  b->zchunk = rc ? saved_zc : best_zc;
  b->dirty = true;
  if (rc) return rc;
  if (tile) *tile = b->tile + 1;
  if (zchunk) *zchunk = b->zchunk;
  return SC_OK;
}

int sc_batch_info(sc_batch* b, int32_t* members, int64_t* items, size_t* free_bytes, size_t* largest_free,
                  int32_t* tile, int32_t* zchunk) {
  if (!b) return fail(SC_EINVAL, "NULL batch");
  int n = 0;
  for (const auto& m : b->members) n += m.h != nullptr;
  if (members) *members = n;
  if (b->tile < 0 && n > 0) { b->tile = batch_default_tile(b); b->dirty = true; }
  if (n > 0) {
    int rc = batch_build(b);
    if (rc) return rc;
  }
  if (items) *items = n > 0 ? b->nitems : 0;
  if (free_bytes) *free_bytes = b->alloc.free_bytes();
  if (largest_free) *largest_free = b->alloc.largest();
  if (tile) *tile = b->tile + 1;
  if (zchunk) *zchunk = b->zchunk;
  return SC_OK;
}

int sc_batch_sync(sc_batch* b) {
  if (!b) return fail(SC_EINVAL, "NULL batch");
  CK(cudaStreamSynchronize(b->stream));
  return SC_OK;
}

}  // extern "C"
