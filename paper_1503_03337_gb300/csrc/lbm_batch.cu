// Batched stepping of many independent domains (C-ABI lbm_batch_*).
//
// Domains of different sizes, Q, storage types and step counters live in one
// batch.  A device table holds one descriptor per active domain and the
// prefix sums of its tiles (a tile is one CTA's block of cells), so a single
// kernel launch advances every domain: CTAs take tiles round-robin across
// all domains, and each tile runs the same per-cell update as the
// single-domain kernel, at its own domain's parity and force time level.
//
// Grouped mode (default): every step launches one kernel per group of
// domains sharing Q, storage, rounding and parity; each is the single-domain
// update specialised at compile time plus a per-CTA domain lookup.  A domain
// big enough to fill the device by itself, or alone in its group, (solo)
// gets its own launch of the single-domain update instead, so batching costs
// it nothing.  Domains are packed into L2-sized clusters that run a block of
// steps each in turn, keeping a cluster's populations in L2 from step to
// step.  Every domain's force and rounding key for the steps ahead are
// computed once per domain and step by a small prepare kernel.
// Persistent mode: one cooperative launch runs `chunk` steps of all domains,
// with a grid barrier between steps (the in-place AA update needs every cell
// of step s done before step s+1 reads its neighbours).  The barrier spins a
// bounded number of times; on time-out it raises a flag, every CTA returns,
// and the host reports LBM_ETIMEOUT.  Population loads go through L2 only
// (ld.cg), because L1 is not coherent between SMs across the steps of one
// launch.  Either way the launches of a chunk are captured once in a CUDA
// graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <tuple>
#include <vector>


#include "lbm_batch.cuh"

namespace lbm {
namespace batchk {
namespace {

// Force F(t_n) and rounding key of entry k at steps n .. n + ns - 1, where n
// is its counter plus s0 (Eq. wa's cosine, evaluated in FP64 and rounded
// once, as the single-domain path does on the host).
__global__ void k_batch_prepare(const BatchEntry* __restrict__ ents, int nent, int s0, int ns,
                                StepDyn* dyn, int stride) {
  const int total = nent * ns;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
    const int k = q % nent, s = q / nent;
    const BatchEntry& e = ents[k];
    const int64_t n = e.n + s0 + s;
    const double c = e.period > 0.0 ? cos(2.0 * M_PI * (double)n / e.period) : 1.0;
    StepDyn v;
    for (int a = 0; a < 3; ++a) v.F[a] = float(e.force[a] * c);
    v.key = step_key(n);
    dyn[(size_t)s * stride + k] = v;
  }
}

// After a chunk: advance every domain's step counter and publish the
// barrier's time-out flag to the host.
__global__ void k_batch_advance(BatchEntry* ents, int nent, int nsteps, const GridBarrier* bar,
                                int* host_flag) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nent; k += gridDim.x * blockDim.x)
    ents[k].n += nsteps;
  if (blockIdx.x == 0 && threadIdx.x == 0 && bar->timed_out) *host_flag = 1;
}

}  // namespace
}  // namespace batchk
}  // namespace lbm

using namespace lbm::batchk;

using namespace lbm;

struct BatchSlot {
  bool used = false;
  DomainDesc dd{};
  lbm_geom geom{};
  lbm_params params{};
  int64_t n = 0;
  size_t fbytes = 0;
  double* u_prev = nullptr;
  int have_prev = 0;
  int64_t prev_step = -1;
  bool has_last = false;  // `last` holds the statistics of a reduction
  lbm_stats last{};
};

struct lbm_batch {
  int device = 0;
  cudaStream_t stream = nullptr;
  int capacity = 0;
  int64_t budget = 0, used_bytes = 0;
  std::vector<BatchSlot> slots;
  // device state
  BatchEntry* ents = nullptr;
  GridBarrier* bar = nullptr;
  int* flag_host = nullptr;  // mapped pinned: barrier timed out
  int* flag_dev = nullptr;
  double* partials = nullptr;
  double* stats_host = nullptr;  // mapped pinned, kNumStats per slot
  double* stats_dev = nullptr;
  BatchEntry* table_host = nullptr;  // pinned staging of the descriptor table
  StepDyn* dyn = nullptr;  // kDynSteps x capacity: force and key per step and entry
  cudaEvent_t table_done = nullptr;  // its last upload has been read
  // launch
  int bx = 64, by = 2;
  int persistent = 0;
  bool has_sr = false;  // some domain rounds stochastically (grouped mode only)
  int grid = 0;      // CTAs of one persistent (cooperative) launch
  int resident = 0;  // CTAs of the grouped kernels resident at once
  int tiles_per_cta = 0;        // grouped launches; 0: automatic
  int64_t solo_min_cells = 0;   // 0: automatic; < 0: no solo domains
  int64_t cluster_bytes = 0;    // L2 cluster budget; 0: automatic; < 0: one cluster
  int64_t l2_bytes = 0;         // the device's L2 size
  long long spin_limit = 1ll << 26;
  int extra_arrivals = 0;
  // table: entries sorted by group; in persistent mode one run over all
  bool dirty = true;
  int nent = 0;
  int64_t total_tiles = 0;
  std::vector<int> order;  // slot of each entry
  struct Group {
    int cluster;                        // L2 cluster (groups are sorted by it)
    int Q, storage, sr, force, parity;  // parity of the domains' step counters
    int solo;                           // one launch per entry
    int first, count;                   // entries
    int64_t tiles;
  };
  std::vector<Group> groups;
  int nclusters = 0;
  std::vector<BatchEntry> host_ents;  // the uploaded table (group-local half)
  // graph of one chunk; captured when a table version runs its third chunk
  // (membership changes invalidate it; a serving loop changes membership
  // every check or two, and a capture replayed once or twice costs more
  // host time than the direct launches it replaces)
  cudaGraphExec_t graph = nullptr;
  int graph_chunk = 0;
  bool graph_ok = true;
  int chunks_this_version = 0;
};

namespace {

constexpr int kDynSteps = 32;  // steps of force/key computed per prepare launch

int bfail(int code, const std::string& m) {
  set_last_error(m);
  return code;
}
int bcuda(cudaError_t e, const char* where) {
  set_last_error(std::string(where) + ": " + cudaGetErrorString(e));
  return LBM_ECUDA;
}

size_t storage_size(int s) {
  return s == LBM_STORAGE_F64 ? 8 : s == LBM_STORAGE_F32 ? 4 : 2;
}

void drop_graph(lbm_batch* b) {
  if (b->graph) cudaGraphExecDestroy(b->graph);
  b->graph = nullptr;
  b->graph_chunk = 0;
}

int fill_desc(const lbm_desc* desc, const lbm_geom* g, const lbm_params* p, DomainDesc& dd) {
  if (desc->Q != 14 && desc->Q != 18)
    return bfail(LBM_EINVAL, "Q must be 14 or 18 (the batch path has no iD3Q26 kernels)");
  if (desc->nx < 1 || desc->ny < 1 || desc->nz < 1)
    return bfail(LBM_EINVAL, "grid sizes must be >= 1");
  if (desc->storage != LBM_STORAGE_F32 && desc->storage != LBM_STORAGE_F16 &&
      desc->storage != LBM_STORAGE_BF16)
    return bfail(LBM_EINVAL, "batched domains store FP32, FP16 or BF16");
  const int64_t N = (int64_t)desc->nx * desc->ny * desc->nz;
  if (N * desc->Q >= (int64_t(1) << 31) || desc->nz > 65535)
    return bfail(LBM_EINVAL, "domain too large (Q*N must be < 2^31)");
  dd = DomainDesc{};
  dd.Q = desc->Q;
  dd.nx = desc->nx;
  dd.ny = desc->ny;
  dd.nz = desc->nz;
  dd.storage = desc->storage;
  dd.N = N;
  if (const char* why = set_faces(dd, g)) return bfail(LBM_EINVAL, why);
  if (dd.neq_vel | dd.neq_pre)
    return bfail(LBM_EINVAL, "extrapolation faces are for single-domain handles only");
  double s[6] = {p->s_c, p->s_e, p->s_q, p->s_nu, p->s_pi, p->s_t};
  if (p->nu > 0.0) s[3] = 1.0 / (3.0 * p->nu + 0.5);
  if (desc->Q == 14) s[4] = s[1];
  for (int k = 0; k < 6; ++k)
    if (!(s[k] > 0.0 && s[k] < 2.0)) return bfail(LBM_EINVAL, "relaxation rates must lie in (0, 2)");
  for (int k = 0; k < 6; ++k) dd.s[k] = s[k];
  for (int k = 0; k < 3; ++k) dd.force[k] = p->force[k];
  if (!std::isfinite(p->force_period) || !std::isfinite(p->p_ref))
    return bfail(LBM_EINVAL, "force period and p_ref must be finite");
  dd.period = p->force_period;
  dd.p_ref = p->p_ref;
  if (p->rounding != LBM_ROUND_NEAREST && p->rounding != LBM_ROUND_STOCHASTIC)
    return bfail(LBM_EINVAL, "unknown rounding mode");
  dd.rounding = p->rounding;
  return LBM_OK;
}

int64_t solo_threshold(const lbm_batch* b) {
  if (b->solo_min_cells < 0) return INT64_MAX;
  if (b->solo_min_cells > 0) return b->solo_min_cells;
  // two full waves of resident CTAs
  return 2 * (int64_t)std::max(1, b->resident) * b->bx * b->by;
}

int64_t cluster_budget(const lbm_batch* b) {
  if (b->cluster_bytes < 0) return INT64_MAX;
  if (b->cluster_bytes > 0) return b->cluster_bytes;
  // half of L2: a cluster's populations stay resident across the steps it
  // runs back to back (measured on a mix of 15-75 MB domains: budgets of a
  // quarter to a half of L2 run 16 % faster than three quarters)
  return b->l2_bytes > 0 ? b->l2_bytes / 2 : (int64_t)64 << 20;
}

// L2 clusters: the active domains packed first-fit, largest first, into sets
// whose population bytes fit the cluster budget (a larger domain is a
// cluster of its own).  A chunk runs its steps in blocks of up to kDynSteps;
// within a block the clusters run one after another, each for all the
// block's steps, so a cluster's populations stay in L2 from step to step.
// Domains are independent, so the order changes no result.
std::vector<int> assign_clusters(lbm_batch* b, const std::vector<int>& idx) {
  const int64_t budget = cluster_budget(b);
  std::vector<int> by_size = idx;
  std::stable_sort(by_size.begin(), by_size.end(), [&](int a, int c) {
    return b->slots[a].fbytes > b->slots[c].fbytes;
  });
  std::vector<int64_t> used;
  std::vector<int> cluster(b->slots.size(), 0);
  for (int i : by_size) {
    const int64_t f = (int64_t)b->slots[i].fbytes;
    int c = -1;
    for (int k = 0; k < (int)used.size(); ++k)
      if (used[k] + f <= budget) {
        c = k;
        break;
      }
    if (c < 0) {
      c = (int)used.size();
      used.push_back(0);
    }
    used[c] += f;
    cluster[i] = c;
  }
  b->nclusters = (int)used.size();
  return cluster;
}

// Rebuild and upload the descriptor table of the active domains, sorted into
// groups of equal (cluster, Q, storage, rounding, force, parity, solo).  A
// domain runs solo (its own launch of the single-domain update) when it is
// big enough to fill the device or has no partner in its group.  Tile prefix
// sums restart at zero in every group (grouped launches) and the persistent
// kernel, which walks all entries, gets its own running prefix in a second
// table half.
int upload_table(lbm_batch* b) {
  std::vector<int> idx;
  for (int i = 0; i < (int)b->slots.size(); ++i)
    if (b->slots[i].used) idx.push_back(i);
  const int64_t solo_min = solo_threshold(b);
  const std::vector<int> cluster = assign_clusters(b, idx);
  auto base_key = [&](int i) {
    const BatchSlot& s = b->slots[i];
    const int sr = s.dd.rounding == LBM_ROUND_STOCHASTIC && s.dd.storage != LBM_STORAGE_F32;
    const int force = s.dd.force[0] != 0.0 || s.dd.force[1] != 0.0 || s.dd.force[2] != 0.0;
    return std::make_tuple(cluster[i], s.dd.Q, s.dd.storage, sr, force, (int)(s.n & 1));
  };
  std::map<decltype(base_key(0)), int> partners;
  for (int i : idx)
    if (b->slots[i].dd.N < solo_min) partners[base_key(i)] += 1;
  auto key = [&](int i) {
    const auto k = base_key(i);
    const auto it = partners.find(k);
    const int solo = b->slots[i].dd.N >= solo_min || it == partners.end() || it->second < 2;
    return std::tuple_cat(k, std::make_tuple(solo));
  };
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int c) { return key(a) < key(c); });
  std::vector<BatchEntry> ents;
  b->order.clear();
  b->groups.clear();
  int64_t tiles = 0;
  for (int i : idx) {
    const BatchSlot& s = b->slots[i];
    BatchEntry e{};
    const double zero[3] = {0.0, 0.0, 0.0};
    e.d = to_domain<float>(s.dd, zero);
    e.Q = s.dd.Q;
    e.storage = s.dd.storage;
    e.rounding = s.dd.rounding;
    e.tiles_x = (s.dd.nx + b->bx - 1) / b->bx;
    e.tiles_y = (s.dd.ny + b->by - 1) / b->by;
    e.tile_begin = tiles;
    e.n = s.n;
    for (int k = 0; k < 3; ++k) e.force[k] = s.dd.force[k];
    e.period = s.dd.period;
    const int64_t nt = (int64_t)e.tiles_x * e.tiles_y * s.dd.nz;
    tiles += nt;
    const auto k = key(i);
    if (b->groups.empty() ||
        std::make_tuple(b->groups.back().cluster, b->groups.back().Q, b->groups.back().storage,
                        b->groups.back().sr, b->groups.back().force, b->groups.back().parity,
                        b->groups.back().solo) != k) {
      b->groups.push_back({std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k),
                           std::get<4>(k), std::get<5>(k), std::get<6>(k), (int)ents.size(), 0,
                           0});
    }
    ents.push_back(e);
    b->groups.back().count += 1;
    b->groups.back().tiles += nt;
    b->order.push_back(i);
  }
  b->nent = (int)ents.size();
  b->total_tiles = tiles;
  b->has_sr = false;
  for (const auto& g : b->groups) b->has_sr = b->has_sr || g.sr;
  // second half: the same entries with tile_begin local to their group
  std::vector<BatchEntry> local = ents;
  for (const auto& g : b->groups) {
    int64_t t = 0;
    for (int k = g.first; k < g.first + g.count; ++k) {
      local[k].tile_begin = t;
      t += (int64_t)local[k].tiles_x * local[k].tiles_y * local[k].d.nz;
    }
  }
  if (!ents.empty()) {
    // the pinned staging area may still be read by the previous upload
    cudaError_t e = cudaEventSynchronize(b->table_done);
    if (e == cudaSuccess) {
      std::memcpy(b->table_host, ents.data(), sizeof(BatchEntry) * ents.size());
      std::memcpy(b->table_host + b->capacity, local.data(), sizeof(BatchEntry) * local.size());
      e = cudaMemcpyAsync(b->ents, b->table_host, sizeof(BatchEntry) * ents.size(),
                          cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b->ents + b->capacity, b->table_host + b->capacity,
                          sizeof(BatchEntry) * local.size(), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(b->table_done, b->stream);
    if (e != cudaSuccess) return bcuda(e, "batch table upload");
  }
  b->host_ents = local;
  b->dirty = false;
  b->chunks_this_version = 0;
  drop_graph(b);
  return LBM_OK;
}

int resident_for_group(lbm_batch* b) {
  int per_sm = group_blocks_per_sm(b->bx * b->by), sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 152 * 4;
  }
  return per_sm * sms;
}

int grid_for_batch(lbm_batch* b) {
  int per_sm = persistent_blocks_per_sm(b->bx * b->by), sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * sms;
}

// Step s (of the chunk) of one group: one launch per solo entry, or one
// grouped launch.
cudaError_t launch_group_step(lbm_batch* b, const lbm_batch::Group& g, int s,
                              const BatchEntry* local, dim3 block) {
  const StepDyn* dyn = b->dyn + (size_t)(s % kDynSteps) * b->capacity;
  const bool odd = ((g.parity + s) & 1) != 0;
  if (g.solo) {
    for (int k = g.first; k < g.first + g.count; ++k) {
      const BatchEntry& he = b->host_ents[k];
      const int periodic = he.period > 0.0;
      SoloLaunch sl{g.storage, g.sr, g.force, odd ? 1 : 0, periodic,
                    dim3(he.tiles_x, he.tiles_y, he.d.nz), block, b->stream, he.d, dyn + k};
      if (!periodic)  // constant force in the descriptor
        for (int a = 0; a < 3; ++a) sl.d.F[a] = float(he.force[a]);
      cudaError_t e = g.Q == 14 ? launch_solo_q14(sl) : launch_solo_q18(sl);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  // contiguous runs of tiles per CTA, short enough to leave about eight
  // waves of CTAs (a partly filled last wave then costs little) and, in big
  // groups, long enough to spread each descriptor load over several tiles
  int per = b->tiles_per_cta;
  if (per < 1) {
    const int64_t waves = std::max<int64_t>(1, (int64_t)b->resident * 8);
    per = (int)std::min<int64_t>(16, std::max<int64_t>(1, g.tiles / waves));
  }
  const unsigned grid = (unsigned)((g.tiles + per - 1) / per);
  GroupLaunch gl{g.storage,       g.sr,          g.force, odd ? 1 : 0, dim3(grid), block,
                 b->stream,       local + g.first, dyn + g.first, g.count, (int)g.tiles, per};
  return g.Q == 14 ? launch_group_q14(gl) : launch_group_q18(gl);
}

// Queue one chunk of `chunk` steps (no graph).
cudaError_t enqueue_chunk(lbm_batch* b, int chunk) {
  dim3 block(b->bx, b->by, 1);
  if (b->persistent && !b->has_sr) {
    cudaError_t e = cudaMemsetAsync(b->bar, 0, sizeof(GridBarrier) - sizeof(int), b->stream);
    if (e != cudaSuccess) return e;
    PersistentLaunch p{b->ents, b->nent, b->total_tiles, chunk,
                       (int)std::max<int64_t>(1, (b->total_tiles + b->grid - 1) / b->grid),
                       b->bar, b->spin_limit, dim3(b->grid), block, b->stream};
    e = launch_persistent(p);
    if (e != cudaSuccess) return e;
  } else {
    const BatchEntry* local = b->ents + b->capacity;
    for (int s0 = 0; s0 < chunk; s0 += kDynSteps) {
      const int ns = std::min(kDynSteps, chunk - s0);
      const int total = b->nent * ns;
      const int blocks = std::min(1024, (total + 255) / 256);
      k_batch_prepare<<<blocks, 256, 0, b->stream>>>(local, b->nent, s0, ns, b->dyn,
                                                     b->capacity);
      size_t g0 = 0;
      while (g0 < b->groups.size()) {  // one cluster: groups g0 .. g1-1
        size_t g1 = g0;
        while (g1 < b->groups.size() && b->groups[g1].cluster == b->groups[g0].cluster) ++g1;
        for (int s = s0; s < s0 + ns; ++s)
          for (size_t gi = g0; gi < g1; ++gi)
            if (cudaError_t e = launch_group_step(b, b->groups[gi], s, local, block))
              return e;
        g0 = g1;
      }
    }
  }
  k_batch_advance<<<1, 256, 0, b->stream>>>(b->ents, b->nent, chunk, b->bar, b->flag_dev);
  k_batch_advance<<<1, 256, 0, b->stream>>>(b->ents + b->capacity, b->nent, chunk, b->bar,
                                            b->flag_dev);
  return cudaGetLastError();
}

}  // namespace

extern "C" {

int lbm_batch_create(int32_t capacity, int64_t budget_bytes, void* cuda_stream, lbm_batch** out) {
  if (!out) return bfail(LBM_EINVAL, "null output");
  *out = nullptr;
  if (capacity < 1 || capacity > 65536) return bfail(LBM_EINVAL, "capacity must be 1..65536");
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return bfail(LBM_ENOMEM, "host allocation failed");
  cudaError_t e = cudaGetDevice(&b->device);
  b->stream = static_cast<cudaStream_t>(cuda_stream);
  b->capacity = capacity;
  b->budget = budget_bytes > 0 ? budget_bytes : INT64_MAX;
  b->slots.resize(capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->ents, 2 * sizeof(BatchEntry) * capacity);
  if (e == cudaSuccess) e = cudaMalloc(&b->bar, sizeof(GridBarrier));
  if (e == cudaSuccess) e = cudaMalloc(&b->partials, sizeof(double) * kReduceBlocks * kNumStats);
  if (e == cudaSuccess) e = cudaHostAlloc(&b->flag_host, sizeof(int), cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&b->flag_dev, b->flag_host, 0);
  if (e == cudaSuccess)
    e = cudaHostAlloc(&b->stats_host, sizeof(double) * kNumStats * capacity, cudaHostAllocMapped);
  if (e == cudaSuccess) e = cudaHostGetDevicePointer(&b->stats_dev, b->stats_host, 0);
  if (e == cudaSuccess)
    e = cudaHostAlloc(&b->table_host, 2 * sizeof(BatchEntry) * capacity, cudaHostAllocDefault);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->table_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&b->dyn, sizeof(StepDyn) * kDynSteps * capacity);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->bar, 0, sizeof(GridBarrier), b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    lbm_batch_destroy(b);
    return bfail(LBM_ENOMEM, "batch allocation failed");
  }
  *b->flag_host = 0;
  b->grid = grid_for_batch(b);
  b->resident = resident_for_group(b);
  int l2 = 0;
  if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, b->device) == cudaSuccess)
    b->l2_bytes = l2;
  cudaGetLastError();
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  drop_graph(b);
  for (BatchSlot& s : b->slots) {
    if (s.dd.f) cudaFree(s.dd.f);
    if (s.u_prev) cudaFree(s.u_prev);
  }
  if (b->ents) cudaFree(b->ents);
  if (b->bar) cudaFree(b->bar);
  if (b->partials) cudaFree(b->partials);
  if (b->flag_host) cudaFreeHost(b->flag_host);
  if (b->stats_host) cudaFreeHost(b->stats_host);
  if (b->table_host) cudaFreeHost(b->table_host);
  if (b->table_done) cudaEventDestroy(b->table_done);
  if (b->dyn) cudaFree(b->dyn);
  delete b;
}

int lbm_batch_add(lbm_batch* b, const lbm_desc* desc, const lbm_geom* geom,
                  const lbm_params* params, int32_t* slot_out) {
  if (!b || !desc || !geom || !params || !slot_out) return bfail(LBM_EINVAL, "null argument");
  DomainDesc dd;
  if (int rc = fill_desc(desc, geom, params, dd)) return rc;
  int slot = -1;
  for (int i = 0; i < b->capacity; ++i)
    if (!b->slots[i].used) {
      slot = i;
      break;
    }
  if (slot < 0) return bfail(LBM_EBUSY, "no free slot");
  const size_t fbytes = (size_t)dd.N * dd.Q * storage_size(dd.storage);
  if (b->used_bytes + (int64_t)fbytes > b->budget) return bfail(LBM_EBUSY, "memory budget exhausted");
  void* f = nullptr;
  cudaError_t e = cudaMallocAsync(&f, fbytes, b->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(f, 0, fbytes, b->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (f) cudaFreeAsync(f, b->stream);
    return bfail(LBM_ENOMEM, "population allocation failed");
  }
  dd.f = f;
  BatchSlot& s = b->slots[slot];
  s = BatchSlot{};
  s.used = true;
  s.dd = dd;
  s.geom = *geom;
  s.params = *params;
  s.fbytes = fbytes;
  b->used_bytes += (int64_t)fbytes;
  b->dirty = true;
  *slot_out = slot;
  return LBM_OK;
}

static int check_slot(lbm_batch* b, int32_t slot) {
  if (!b) return bfail(LBM_EINVAL, "null batch");
  if (slot < 0 || slot >= b->capacity || !b->slots[slot].used)
    return bfail(LBM_EINVAL, "no domain in that slot");
  return LBM_OK;
}

int lbm_batch_remove(lbm_batch* b, int32_t slot) {
  if (int rc = check_slot(b, slot)) return rc;
  BatchSlot& s = b->slots[slot];
  cudaFreeAsync(s.dd.f, b->stream);
  if (s.u_prev) cudaFreeAsync(s.u_prev, b->stream);
  b->used_bytes -= (int64_t)s.fbytes;
  s = BatchSlot{};
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_init_equilibrium(lbm_batch* b, int32_t slot, const double* u, const double* p,
                               int on_device) {
  if (int rc = check_slot(b, slot)) return rc;
  if (!on_device && (u || p)) return bfail(LBM_EINVAL, "batch init takes device arrays");
  BatchSlot& s = b->slots[slot];
  cudaError_t e = launch_init(s.dd, u, p, b->stream);
  if (e != cudaSuccess) return bcuda(e, "init kernel");
  s.n = 0;
  s.have_prev = 0;
  s.prev_step = -1;
  s.has_last = false;
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_step(lbm_batch* b, int64_t nsteps, int32_t chunk) {
  if (!b) return bfail(LBM_EINVAL, "null batch");
  if (nsteps < 0) return bfail(LBM_EINVAL, "nsteps < 0");
  if (*static_cast<volatile int*>(b->flag_host))
    return bfail(LBM_ETIMEOUT, "a grid barrier of an earlier batch launch timed out");
  if (b->dirty)
    if (int rc = upload_table(b)) return rc;
  if (b->nent == 0 || nsteps == 0) return LBM_OK;
  if (chunk < 1) chunk = 1;
  if (b->persistent && b->grid < 1) b->persistent = 0;
  int64_t left = nsteps;
  while (left > 0) {
    const int c = (int)std::min<int64_t>(left, chunk);
    cudaError_t e = cudaSuccess;
    if (c == chunk && b->graph_ok && (b->graph || b->chunks_this_version >= 2)) {
      if (!b->graph || b->graph_chunk != c) {
        drop_graph(b);
        cudaGraph_t g = nullptr;
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaError_t e1 = enqueue_chunk(b, c);
          e = cudaStreamEndCapture(b->stream, &g);
          if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {  // capture not possible here: launch directly
          cudaGetLastError();
          b->graph_ok = false;
          b->graph = nullptr;
        } else {
          b->graph_chunk = c;
        }
      }
      if (b->graph) e = cudaGraphLaunch(b->graph, b->stream);
      else e = enqueue_chunk(b, c);
    } else {
      e = enqueue_chunk(b, c);
    }
    if (e != cudaSuccess) return bcuda(e, "batch step");
    for (int k : b->order) b->slots[k].n += c;
    left -= c;
    b->chunks_this_version += 1;
    // grouped launches key on parity: an odd chunk flips every group's parity
    if (c & 1) {
      for (auto& g : b->groups) g.parity ^= 1;
      drop_graph(b);
    }
  }
  return LBM_OK;
}

int lbm_batch_get_step(lbm_batch* b, int32_t slot, int64_t* n) {
  if (int rc = check_slot(b, slot)) return rc;
  if (!n) return bfail(LBM_EINVAL, "null output");
  *n = b->slots[slot].n;
  return LBM_OK;
}

int lbm_batch_read_fields(lbm_batch* b, int32_t slot, unsigned mask, void* dst,
                          int dst_on_device, int dtype) {
  if (int rc = check_slot(b, slot)) return rc;
  if (!dst || !dst_on_device) return bfail(LBM_EINVAL, "batch read-back takes a device buffer");
  if (mask == 0 || (mask & ~7u)) return bfail(LBM_EINVAL, "bad field mask");
  if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return bfail(LBM_EINVAL, "bad dtype");
  BatchSlot& s = b->slots[slot];
  cudaError_t e = launch_read(s.dd, s.n, mask, dst, dtype, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch read");
  return LBM_OK;
}

// Queue the FP64 reductions of one slot into its stats area.
static int queue_reduction(lbm_batch* b, int32_t slot) {
  BatchSlot& s = b->slots[slot];
  if (!s.u_prev) {
    cudaError_t e = cudaMallocAsync(&s.u_prev, sizeof(double) * 3 * s.dd.N, b->stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      s.u_prev = nullptr;
      return bfail(LBM_ENOMEM, "snapshot allocation failed");
    }
    s.have_prev = 0;
  }
  cudaError_t e = launch_reduce(s.dd, s.n, s.u_prev, s.have_prev, b->partials,
                                b->stats_dev + (size_t)slot * kNumStats, b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch reduction");
  return LBM_OK;
}

// Statistics of a slot whose reduction has completed; the snapshot is now
// the current velocity.
static void take_stats(lbm_batch* b, int32_t slot, lbm_stats* out) {
  BatchSlot& s = b->slots[slot];
  const double* v = b->stats_host + (size_t)slot * kNumStats;
  out->step = s.n;
  out->prev_step = s.have_prev ? s.prev_step : -1;
  for (int k = 0; k < 3; ++k) {
    out->sum_abs_du[k] = v[k];
    out->sum_abs_u[k] = v[3 + k];
    out->sum_abs_u_prev[k] = v[6 + k];
    out->sum_u[k] = v[10 + k];
  }
  out->sum_P = v[9];
  out->nonfinite = (int64_t)v[kNumSums - 1];
  out->max_abs_u = v[kNumSums];
  s.have_prev = 1;
  s.prev_step = s.n;
  s.last = *out;
  s.has_last = true;
}

int lbm_batch_reductions(lbm_batch* b, int32_t slot, lbm_stats* out) {
  if (int rc = check_slot(b, slot)) return rc;
  if (!out) return bfail(LBM_EINVAL, "null output");
  if (int rc = queue_reduction(b, slot)) return rc;
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch reduction");
  take_stats(b, slot, out);
  return LBM_OK;
}

int lbm_batch_reductions_all(lbm_batch* b, lbm_stats* out, int32_t* slots, int32_t* count) {
  if (!b || !out || !slots || !count) return bfail(LBM_EINVAL, "null argument");
  int n = 0;
  for (int i = 0; i < b->capacity; ++i)
    if (b->slots[i].used) {
      if (int rc = queue_reduction(b, i)) return rc;
      slots[n++] = i;
    }
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch reductions");
  for (int k = 0; k < n; ++k) take_stats(b, slots[k], &out[k]);
  *count = n;
  return LBM_OK;
}

int lbm_batch_residual(lbm_batch* b, int32_t slot, int32_t kind, int32_t component, double* r) {
  if (int rc = check_slot(b, slot)) return rc;
  if (!b->slots[slot].has_last) return bfail(LBM_EINVAL, "no reduction of this slot yet");
  return lbm_stats_residual(&b->slots[slot].last, kind, component, r);
}

int lbm_batch_set_launch(lbm_batch* b, int32_t bx, int32_t by, int32_t persistent) {
  if (!b) return bfail(LBM_EINVAL, "null batch");
  if (bx < 32 || bx % 32 != 0 || by < 1 || (int64_t)bx * by > 256)
    return bfail(LBM_EINVAL, "block must be bx (multiple of 32) x by with bx*by <= 256");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch set_launch");
  b->bx = bx;
  b->by = by;
  b->persistent = persistent ? 1 : 0;
  b->grid = grid_for_batch(b);
  b->resident = resident_for_group(b);
  b->graph_ok = true;
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_set_schedule(lbm_batch* b, int32_t tiles_per_cta, int64_t solo_min_cells,
                           int64_t cluster_bytes) {
  if (!b) return bfail(LBM_EINVAL, "null batch");
  if (tiles_per_cta < 0 || tiles_per_cta > 4096) return bfail(LBM_EINVAL, "tiles_per_cta must be 0..4096");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "batch set_schedule");
  b->tiles_per_cta = tiles_per_cta;
  b->solo_min_cells = solo_min_cells;
  b->cluster_bytes = cluster_bytes;
  b->dirty = true;
  return LBM_OK;
}

int lbm_batch_info(lbm_batch* b, int32_t* active, int64_t* used_bytes, int64_t* total_cells) {
  if (!b) return bfail(LBM_EINVAL, "null batch");
  int n = 0;
  int64_t cells = 0;
  for (const BatchSlot& s : b->slots)
    if (s.used) {
      ++n;
      cells += s.dd.N;
    }
  if (active) *active = n;
  if (used_bytes) *used_bytes = b->used_bytes;
  if (total_cells) *total_cells = cells;
  return LBM_OK;
}

int lbm_batch_set_barrier_test(lbm_batch* b, int32_t extra_arrivals, int64_t spin_limit) {
  if (!b) return bfail(LBM_EINVAL, "null batch");
  if (extra_arrivals < 0 || spin_limit < 1) return bfail(LBM_EINVAL, "bad barrier test values");
  cudaError_t e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bcuda(e, "barrier test");
  b->extra_arrivals = extra_arrivals;
  b->spin_limit = spin_limit;
  GridBarrier g{0u, 0u, 0, extra_arrivals};
  e = cudaMemcpy(b->bar, &g, sizeof g, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return bcuda(e, "barrier test");
  *b->flag_host = 0;
  drop_graph(b);
  return LBM_OK;
}

}  // extern "C"
