// Batched ensembles: many independent periodic boxes (replicas) of uneven sizes, seeds,
// relaxation times and thermal energies, all advanced by one persistent kernel launch.
//
// Work items are (step, tile) pairs handed out in step-major order by a global counter;
// a tile is kTile consecutive sites of one replica. Before a CTA updates replica r at
// step t it waits until all tiles of replica r at step t - 1 are complete (a per-replica
// completion counter; this also protects the buffer the step writes, which step t - 1
// read). The earliest unfinished item never waits: its dependencies have smaller queue
// indices and were taken earlier, so the kernel always progresses. Every wait is bounded;
// a CTA that gives up sets the error flag and leaves, which makes the CTAs that wait on
// it give up as well, so the launch ends with an error status instead of hanging.
//
// Population loads bypass L1 (__ldcg): the data were written by other CTAs during the
// same launch. Each replica's arithmetic is the single-box general kernel's, with Philox
// key = the replica's seed and replica word 0, so a replica reproduces its single-box run.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rflbm.h"
#include "rflbm_aux.h"

namespace rflbm_dev {

struct ReplicaDev {
  Geometry geo;
  CollideParams cp;
  StoreScale ss;
  void* buf[2];
  uint32_t key0, key1;
  int noise;          // kT > 0
  int cur;            // buffer holding the state at the start of the launch
  int64_t tile_begin;  // first global tile index of this replica
  int64_t ntiles;
};

constexpr uint32_t kBatchMaxPolls = 1u << 24;

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

template <int kStore, int kTile>
__global__ void __launch_bounds__(kTile) k_batch_run(const ReplicaDev* __restrict__ reps,
                                                     const int* __restrict__ tile_rep,
                                                     int64_t tiles_per_step, int64_t nsteps,
                                                     const unsigned long long* step0_ptr,
                                                     unsigned long long* queue,
                                                     unsigned long long* done, int* err) {
  using S = Storage<kStore>;
  using T = typename S::T;
  __shared__ unsigned long long next_sh;
  __shared__ int fail_sh;
  const int64_t total = tiles_per_step * nsteps;
  const uint32_t step0 = (uint32_t)*step0_ptr;
  if (threadIdx.x == 0) next_sh = atomicAdd(queue, 1ull);
  __syncthreads();
  unsigned long long item = next_sh;
  while ((int64_t)item < total) {
    const int64_t t = (int64_t)item / tiles_per_step;
    const int64_t j = (int64_t)item - t * tiles_per_step;
    const int r = __ldg(tile_rep + j);
    const ReplicaDev& rep = reps[r];  // uniform over the CTA: read through the read-only cache
    if (threadIdx.x == 0) {
      // the next item is taken now and published by the barrier below
      next_sh = atomicAdd(queue, 1ull);
      int failed = 0;
      if (t > 0) {
        const unsigned long long need = (unsigned long long)(t * rep.ntiles);
        uint32_t it = 0;
        while (ld_acquire(&done[r]) < need) {
          if (++it >= kBatchMaxPolls) {
            failed = 1;
            break;
          }
          __nanosleep(64);
        }
      }
      fail_sh = failed;
    }
    __syncthreads();  // the dependency holds for the whole CTA; next_sh and fail_sh are set
    const unsigned long long next = next_sh;
    if (fail_sh) {
      if (threadIdx.x == 0) atomicOr(err, 1);
      return;
    }
    const int parity = (rep.cur + (int)(t & 1)) & 1;
    const T* src = static_cast<const T*>(rep.buf[parity]);
    T* dst = static_cast<T*>(rep.buf[parity ^ 1]);
    const int64_t s64 = (j - rep.tile_begin) * kTile + threadIdx.x;
    if (s64 < (int64_t)rep.geo.n) {
      const uint32_t s = (uint32_t)s64;
      const PullDeltas d = pull_deltas(s, rep.geo);
      float G[3][3][3];
#pragma unroll
      for (int i = 0; i < kQ; ++i)
        G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1] =
            S::load(__ldcg(src + s + pull_delta(d, i) + plane_of(i) * rep.geo.ps), class_of(i), rep.ss);
      SiteNoise noise;
      const uint32_t step = step0 + (uint32_t)t;
      if (rep.noise) {
        site_noise(s, step, 0u, rep.key0, rep.key1, noise);
        collide_site<kModelReg, true, false, false>(G, rep.cp, noise);
      } else {
        collide_site<kModelReg, false, false, false>(G, rep.cp, noise);
      }
#pragma unroll
      for (int i = 0; i < kQ; ++i)
        dst[s + plane_of(i) * rep.geo.ps] = S::store(G[cx_of(i) + 1][cy_of(i) + 1][cz_of(i) + 1], class_of(i), rep.ss);
    }
    __syncthreads();  // every thread's stores of this item precede the release below
    if (threadIdx.x == 0) {
      __threadfence();  // cumulative over the CTA's stores ordered by the barrier
      atomicAdd(&done[r], 1ull);
    }
    item = next;
  }
}

template <int kStore, int kTile>
static cudaError_t launch_batch_t(const ReplicaDev* reps, const int* tile_rep, int64_t tiles,
                                  int64_t nsteps, const unsigned long long* step0, unsigned long long* queue,
                                  unsigned long long* done, int* err, int grid, cudaStream_t st) {
  k_batch_run<kStore, kTile><<<grid, kTile, 0, st>>>(reps, tile_rep, tiles, nsteps, step0, queue, done, err);
  return cudaGetLastError();
}

template <int kStore, int kTile>
static int occupancy_t() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_batch_run<kStore, kTile>, kTile, 0) != cudaSuccess) return 1;
  return std::max(n, 1);
}

static int batch_occupancy(int storage, int tile) {
  switch (storage * 10 + (tile == 128 ? 0 : (tile == 256 ? 1 : 2))) {
    case 0: return occupancy_t<kStoreF32, 128>();
    case 1: return occupancy_t<kStoreF32, 256>();
    case 2: return occupancy_t<kStoreF32, 512>();
    case 10: return occupancy_t<kStoreF16, 128>();
    case 11: return occupancy_t<kStoreF16, 256>();
    case 12: return occupancy_t<kStoreF16, 512>();
    case 20: return occupancy_t<kStoreBF16, 128>();
    case 21: return occupancy_t<kStoreBF16, 256>();
    default: return occupancy_t<kStoreBF16, 512>();
  }
}

static cudaError_t launch_batch(int storage, int tile, const ReplicaDev* reps, const int* tile_rep,
                                int64_t tiles, int64_t nsteps, const unsigned long long* step0,
                                unsigned long long* queue, unsigned long long* done, int* err,
                                int grid, cudaStream_t st) {
#define RFLBM_BATCH_CASE(S, T) \
  return launch_batch_t<S, T>(reps, tile_rep, tiles, nsteps, step0, queue, done, err, grid, st)
  switch (storage * 10 + (tile == 128 ? 0 : (tile == 256 ? 1 : 2))) {
    case 0: RFLBM_BATCH_CASE(kStoreF32, 128);
    case 1: RFLBM_BATCH_CASE(kStoreF32, 256);
    case 2: RFLBM_BATCH_CASE(kStoreF32, 512);
    case 10: RFLBM_BATCH_CASE(kStoreF16, 128);
    case 11: RFLBM_BATCH_CASE(kStoreF16, 256);
    case 12: RFLBM_BATCH_CASE(kStoreF16, 512);
    case 20: RFLBM_BATCH_CASE(kStoreBF16, 128);
    case 21: RFLBM_BATCH_CASE(kStoreBF16, 256);
    default: RFLBM_BATCH_CASE(kStoreBF16, 512);
  }
#undef RFLBM_BATCH_CASE
}

}  // namespace rflbm_dev

using namespace rflbm_dev;

struct rflbm_batch {
  int n = 0;
  int device = 0;
  int num_sms = 1;
  int storage = kStoreF32;
  double rho0 = 1.0;
  cudaStream_t stream = nullptr;
  std::vector<rflbm_replica_t> cfg;
  std::vector<ReplicaDev> host;
  ReplicaDev* dev_reps = nullptr;
  int* tile_rep = nullptr;
  int64_t tiles = 0;
  int tile = 256;
  int ctas_per_sm = 1;
  unsigned long long* counters = nullptr;  // [0] queue, [1 + r] completion per replica
  unsigned long long* step0 = nullptr;     // first step index of the current run (device)
  int* err = nullptr;
  double* partials = nullptr;
  int stat_blocks = 0;
  int64_t step = 0;
  bool initialised = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_steps = -1;
};

namespace {

int bfail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  return record_error(code, buf, nullptr);
}

int bcuda(cudaError_t e, const char* what) {
  return record_error(e == cudaErrorMemoryAllocation ? RFLBM_ENOMEM : RFLBM_ECUDA, what,
                      cudaGetErrorString(e));
}

#define BCUDA(call, what)                       \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return bcuda(e_, what); \
  } while (0)

int64_t pstride(int64_t n) { return (n + 63) / 64 * 64; }

int upload_reps(rflbm_batch* b) {
  BCUDA(cudaMemcpyAsync(b->dev_reps, b->host.data(), sizeof(ReplicaDev) * b->n, cudaMemcpyHostToDevice, b->stream),
        "uploading replica descriptors");
  return RFLBM_OK;
}

// Builds the per-replica descriptors and the tile map for tile size `tile`.
int layout_tiles(rflbm_batch* b, int tile) {
  int64_t tiles = 0;
  for (int r = 0; r < b->n; ++r) {
    b->host[r].tile_begin = tiles;
    b->host[r].ntiles = ((int64_t)b->host[r].geo.n + tile - 1) / tile;
    tiles += b->host[r].ntiles;
  }
  std::vector<int> map((size_t)tiles);
  for (int r = 0; r < b->n; ++r)
    for (int64_t j = 0; j < b->host[r].ntiles; ++j) map[(size_t)(b->host[r].tile_begin + j)] = r;
  cudaFree(b->tile_rep);
  b->tile_rep = nullptr;
  BCUDA(cudaMalloc(&b->tile_rep, sizeof(int) * (size_t)tiles), "allocating the tile map");
  BCUDA(cudaMemcpy(b->tile_rep, map.data(), sizeof(int) * (size_t)tiles, cudaMemcpyHostToDevice), "uploading the tile map");
  b->tiles = tiles;
  b->tile = tile;
  b->ctas_per_sm = batch_occupancy(b->storage, tile);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (b->graph) {
    cudaGraphDestroy(b->graph);
    b->graph = nullptr;
  }
  b->graph_steps = -1;
  return upload_reps(b);
}

// The launch sequence of one run: clear the queue and completion counters, run the
// persistent kernel.
int enqueue_run(rflbm_batch* b, int64_t nsteps, cudaStream_t st) {
  BCUDA(cudaMemsetAsync(b->counters, 0, sizeof(unsigned long long) * (size_t)(b->n + 1), st),
        "clearing the work counters");
  const int64_t items = b->tiles * nsteps;
  const int64_t full = (int64_t)b->ctas_per_sm * b->num_sms;
  const int grid = (int)std::max<int64_t>(1, std::min(full, items));
  BCUDA(launch_batch(b->storage, b->tile, b->dev_reps, b->tile_rep, b->tiles, nsteps, b->step0,
                     b->counters, b->counters + 1, b->err, grid, st),
        "launching the batched step kernel");
  return RFLBM_OK;
}

int bsync(rflbm_batch* b, const char* what) {
  BCUDA(cudaStreamSynchronize(b->stream), what);
  int flag = 0;
  BCUDA(cudaMemcpy(&flag, b->err, sizeof(int), cudaMemcpyDeviceToHost), "reading the error flag");
  if (flag) {
    cudaMemset(b->err, 0, sizeof(int));
    return bfail(RFLBM_ETIMEOUT, "%s: a CTA gave up waiting for a replica's previous step", what);
  }
  return RFLBM_OK;
}

// Runs n steps through a CUDA graph of the launch sequence (captured once per n; the
// starting step is read by the kernel from device memory, written before each launch).
int run_graph(rflbm_batch* b, int64_t n) {
  const unsigned long long s0 = (unsigned long long)b->step;
  BCUDA(cudaMemcpyAsync(b->step0, &s0, sizeof(s0), cudaMemcpyHostToDevice, b->stream), "setting the step index");
  if (!b->exec || b->graph_steps != n) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaStream_t cap;
    BCUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "creating the capture stream");
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    int rc = RFLBM_OK;
    if (e == cudaSuccess) rc = enqueue_run(b, n, cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return bcuda(e, "capturing the batched run");
    if (rc != RFLBM_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e2 != cudaSuccess) return bcuda(e2, "capturing the batched run");
    BCUDA(cudaGraphInstantiate(&b->exec, g, 0), "instantiating the batched run graph");
    b->graph = g;
    b->graph_steps = n;
  }
  BCUDA(cudaGraphLaunch(b->exec, b->stream), "launching the batched run graph");
  return RFLBM_OK;
}

}  // namespace

extern "C" {

rflbm_batch_t* rflbm_batch_create(const rflbm_replica_t* reps, int n, double rho0, int storage,
                                  int tile) {
  if (!reps || n < 1) {
    bfail(RFLBM_EINVAL, "rflbm_batch_create: no replicas");
    return nullptr;
  }
  if (!(rho0 > 0.0) || (storage != RFLBM_STORE_F32 && storage != RFLBM_STORE_F16 && storage != RFLBM_STORE_BF16) ||
      (tile != 0 && tile != 128 && tile != 256 && tile != 512)) {
    bfail(RFLBM_EINVAL, "rflbm_batch_create: invalid rho0, storage or tile");
    return nullptr;
  }
  for (int r = 0; r < n; ++r) {
    rflbm_config_t c;
    rflbm_config_default(&c);
    c.nx = reps[r].nx; c.ny = reps[r].ny; c.nz = reps[r].nz;
    c.tau = reps[r].tau; c.kT = reps[r].kT; c.rho0 = rho0; c.storage = storage;
    if (rflbm_buffer_bytes(&c) < 0) return nullptr;  // validation message already recorded
  }
  rflbm_batch* b = new (std::nothrow) rflbm_batch();
  if (!b) {
    bfail(RFLBM_ENOMEM, "allocating the batch handle");
    return nullptr;
  }
  b->n = n;
  b->rho0 = rho0;
  b->storage = storage == RFLBM_STORE_F16 ? kStoreF16 : (storage == RFLBM_STORE_BF16 ? kStoreBF16 : kStoreF32);
  b->cfg.assign(reps, reps + n);
  b->host.resize(n);
  cudaGetDevice(&b->device);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device);
  const size_t elem = storage_bytes(b->storage);
  int rc = RFLBM_OK;
  for (int r = 0; r < n && rc == RFLBM_OK; ++r) {
    ReplicaDev& d = b->host[r];
    std::memset(&d, 0, sizeof(d));
    const rflbm_replica_t& c = reps[r];
    Geometry& g = d.geo;
    g.nx = c.nx; g.ny = c.ny; g.nz = c.nz;
    g.view = kViewPull;
    g.nxy = (uint32_t)c.nx * (uint32_t)c.ny;
    g.n = (uint32_t)((int64_t)c.nx * c.ny * c.nz);
    g.ps = pstride(g.n);
    g.div_nx = make_fastdiv(g.nx);
    g.div_nxy = make_fastdiv(g.nxy);
    // collision and noise parameters: the single-box handle's (Reg-FLBM, omega_g = 1)
    const double om = 1.0 / c.tau, cs2 = 1.0 / 3.0;
    d.cp.rho0 = (float)rho0;
    d.cp.omega = (float)om;
    d.cp.neq_diag = (float)((1.0 - om) / bnorm(2, 0, 0));
    d.cp.neq_off = (float)((1.0 - om) / bnorm(1, 1, 0));
    d.cp.ghost_keep = 0.0f;
    d.cp.sqrt_rho0 = (float)std::sqrt(rho0);
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q)
        for (int s = 0; s < 3; ++s) {
          if (p + q + s < 2) continue;
          const int k = mode_of(p, q, s);
          const double ok = k < 10 ? om : 1.0;
          d.cp.amp[k - 4] = (float)std::sqrt(c.kT * ok * (2.0 - ok) / (cs2 * bnorm(p, q, s)));
        }
    const double wc[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
    for (int k = 0; k < 4; ++k) {
      if (b->storage == kStoreF32) {
        d.ss.scale[k] = d.ss.inv_scale[k] = 1.0f;
      } else {
        const int e = (int)std::lround(-std::log2(std::sqrt(3.0 * wc[k] * rho0 * std::max(c.kT, 1e-6))));
        d.ss.scale[k] = std::ldexp(1.0f, e);
        d.ss.inv_scale[k] = std::ldexp(1.0f, -e);
      }
    }
    d.key0 = (uint32_t)(c.seed & 0xffffffffu);
    d.key1 = (uint32_t)(c.seed >> 32);
    d.noise = c.kT > 0.0;
    d.cur = 0;
    for (int k = 0; k < 2 && rc == RFLBM_OK; ++k) {
      cudaError_t e = cudaMalloc(&d.buf[k], (size_t)g.ps * kQ * elem);
      if (e == cudaSuccess) e = cudaMemset(d.buf[k], 0, (size_t)g.ps * kQ * elem);
      if (e != cudaSuccess) rc = bcuda(e, "allocating replica populations");
    }
  }
  if (rc == RFLBM_OK) {
    cudaError_t e = cudaMalloc((void**)&b->dev_reps, sizeof(ReplicaDev) * n);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->counters, sizeof(unsigned long long) * (size_t)(n + 2));
    if (e == cudaSuccess) b->step0 = b->counters + n + 1;
    if (e == cudaSuccess) e = cudaMemset(b->step0, 0, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
    if (e != cudaSuccess) rc = bcuda(e, "allocating batch descriptors");
  }
  if (rc == RFLBM_OK) {
    int64_t nmax = 0;
    for (int r = 0; r < n; ++r) nmax = std::max<int64_t>(nmax, b->host[r].geo.n);
    b->stat_blocks = std::max(1, (int)std::min<int64_t>(4 * (int64_t)b->num_sms, (nmax + 255) / 256));
    cudaError_t e = cudaMalloc((void**)&b->partials, sizeof(double) * ((size_t)b->stat_blocks * kStatOutFields + 8));
    if (e != cudaSuccess) rc = bcuda(e, "allocating the reduction scratch");
  }
  if (rc == RFLBM_OK) rc = layout_tiles(b, tile ? tile : 256);
  if (rc == RFLBM_OK && tile == 0) {
    // autotuner: time a few steps of every tile size on this ensemble and keep the fastest
    // (the populations are reset by the init call that must follow)
    cudaEvent_t t0, t1;
    cudaEventCreate(&t0);
    cudaEventCreate(&t1);
    float best = 1e30f;
    int best_tile = 256;
    for (int cand : {128, 256, 512}) {
      if (layout_tiles(b, cand) != RFLBM_OK) continue;
      enqueue_run(b, 1, b->stream);  // warm-up
      cudaEventRecord(t0, b->stream);
      enqueue_run(b, 3, b->stream);
      cudaEventRecord(t1, b->stream);
      float ms = 1e30f;
      if (cudaEventSynchronize(t1) == cudaSuccess) cudaEventElapsedTime(&ms, t0, t1);
      if (ms < best) {
        best = ms;
        best_tile = cand;
      }
    }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    rc = layout_tiles(b, best_tile);
    if (rc == RFLBM_OK) rc = bsync(b, "autotuning the batch");
  }
  if (rc != RFLBM_OK) {
    rflbm_batch_destroy(b);
    return nullptr;
  }
  return b;
}

void rflbm_batch_destroy(rflbm_batch_t* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  for (auto& d : b->host) {
    cudaFree(d.buf[0]);
    cudaFree(d.buf[1]);
  }
  cudaFree(b->dev_reps);
  cudaFree(b->tile_rep);
  cudaFree(b->counters);
  cudaFree(b->err);
  cudaFree(b->partials);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

int rflbm_batch_tuning(const rflbm_batch_t* b, int* tile, int* ctas_per_sm, int64_t* tiles_per_step) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  if (tile) *tile = b->tile;
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  if (tiles_per_step) *tiles_per_step = b->tiles;
  return RFLBM_OK;
}

int rflbm_batch_init_rest(rflbm_batch_t* b) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  for (auto& d : b->host) {
    d.cur = 0;
    BCUDA(cudaMemsetAsync(d.buf[0], 0, (size_t)d.geo.ps * kQ * storage_bytes(b->storage), b->stream),
          "clearing replica populations");
  }
  b->step = 0;
  b->initialised = true;
  if (int e = upload_reps(b)) return e;
  return bsync(b, "rflbm_batch_init_rest");
}

int rflbm_batch_run(rflbm_batch_t* b, int64_t n) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  if (!b->initialised) return bfail(RFLBM_ESTATE, "batch state not initialised (call rflbm_batch_init_rest)");
  if (n < 0) return bfail(RFLBM_EINVAL, "negative step count");
  if (n == 0) return RFLBM_OK;
  if (int e = run_graph(b, n)) return e;
  b->step += n;
  if (n & 1) {
    for (auto& d : b->host) d.cur ^= 1;
    if (int e = upload_reps(b)) return e;
  }
  return RFLBM_OK;
}

int rflbm_batch_synchronize(rflbm_batch_t* b) {
  if (!b) return bfail(RFLBM_EINVAL, "batch handle is NULL");
  return bsync(b, "rflbm_batch_synchronize");
}

int rflbm_batch_get_populations(rflbm_batch_t* b, int r, double* f) {
  if (!b || r < 0 || r >= b->n || !f) return bfail(RFLBM_EINVAL, "invalid batch, replica or output");
  if (!b->initialised) return bfail(RFLBM_ESTATE, "batch state not initialised");
  const ReplicaDev& d = b->host[r];
  double* dev = nullptr;
  const size_t bytes = sizeof(double) * kQ * (size_t)d.geo.n;
  BCUDA(cudaMalloc((void**)&dev, bytes), "allocating the export buffer");
  cudaError_t e = launch_get_populations_f64(d.geo, d.cp.rho0, d.ss, b->storage, d.buf[d.cur], dev, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, dev, bytes, cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  cudaFree(dev);
  if (e != cudaSuccess) return bcuda(e, "exporting replica populations");
  return bsync(b, "rflbm_batch_get_populations");
}

int rflbm_batch_stats(rflbm_batch_t* b, int r, rflbm_stats_t* out) {
  if (!b || r < 0 || r >= b->n || !out) return bfail(RFLBM_EINVAL, "invalid batch, replica or output");
  if (!b->initialised) return bfail(RFLBM_ESTATE, "batch state not initialised");
  const ReplicaDev& d = b->host[r];
  const int blocks = std::max(1, (int)std::min<int64_t>(b->stat_blocks, ((int64_t)d.geo.n + 255) / 256));
  double* res = b->partials + (size_t)b->stat_blocks * kStatOutFields;
  BCUDA(launch_stats(d.geo, d.cp.rho0, d.ss, b->storage, d.buf[d.cur], b->partials, blocks, res, b->stream),
        "launching replica stats");
  double host[kStatOutFields];
  BCUDA(cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, b->stream), "copying replica stats");
  if (int e = bsync(b, "rflbm_batch_stats")) return e;
  out->step = b->step;
  out->mass = (double)d.geo.n * b->rho0 + host[0];
  out->momentum[0] = host[1];
  out->momentum[1] = host[2];
  out->momentum[2] = host[3];
  out->max_speed = host[4];
  out->nonfinite = (int64_t)host[5];
  if (out->nonfinite > 0) return bfail(RFLBM_EUNSTABLE, "replica %d holds non-finite values", r);
  return RFLBM_OK;
}

}  // extern "C"
