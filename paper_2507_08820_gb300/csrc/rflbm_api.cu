// Host side of the C ABI declared in include/rflbm.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cufft.h>

#include "../../include/rflbm.h"
#include "../../include/rflbm_testing.h"
#include "rflbm_aux.h"
#include "rflbm_diag.h"

using namespace rflbm_dev;

struct rflbm {
  rflbm_config_t cfg;
  Geometry geo;
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  void* buf[2] = {nullptr, nullptr};
  size_t elem = 4;             // bytes per stored population value
  StoreScale ss{};             // 16-bit storage scales (ones for float32)
  bool own_buf = false;
  int cur = 0;            // buffer holding the current state (ping-pong)
  bool aa = false;        // AA pattern: one buffer (buf[0]) updated in place
  int phase = 0;          // AA: parity of the steps taken since the state was set
  int64_t step = 0;
  bool initialised = false;
  StepVariant variant{};
  CollideParams cp{};
  double* partials = nullptr;  // stats scratch: kStatOutFields doubles per block + 8 out
  int stat_blocks = 0;
  int* err = nullptr;          // device error flag set by bounded waits in kernels
  int tma_width = 0;           // row-segment width of the TMA step path (0: generic)
  int kernel = RFLBM_KERNEL_GATHER;  // the step kernel in use
  CUtensorMap load_map[2];     // per buffer: source-row loads with halo
  CUtensorMap store_map[2];    // per buffer: row-segment stores
  CUtensorMap row_map;         // AA with one segment per row: three-plane row stores
  uint32_t test_extra_tx = 0;  // testing hook (rflbm_testing_expect_extra_bytes)
  bool has_row_map = false;
  // diagnostics (allocated on first use)
  double* diag_partials = nullptr;
  size_t diag_partials_bytes = 0;
  double* diag_field = nullptr;   // one FP64 field (N)
  void* diag_spec = nullptr;      // its D2Z spectrum
  cufftHandle fft_plan = 0;
  bool fft_ready = false;
  void* staging = nullptr;     // device staging for host<->device transfers
  size_t staging_bytes = 0;
  // z-slab of a decomposed box (cfg.nz_global > 0): ghost rows at both z faces
  bool slab = false;
  int exchange = 0;            // the face exchange the last step requires (kExchange*)
  cudaEvent_t faces_ready = nullptr;  // recorded after the boundary rows of the last step
  cudaEvent_t exchanged = nullptr;    // recorded where the exchange ends
  cudaStream_t halo_stream = nullptr; // copies of rflbm_slab_exchange
};

namespace rflbm_dev {
// The row-segment width for rows that no width divides (rflbm_step_tma.cu), 0 when none.
int tma_ragged_width(uint32_t nx, size_t elem);
}  // namespace rflbm_dev

namespace {

thread_local std::string g_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? RFLBM_ENOMEM : RFLBM_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorString(e), cudaGetErrorName(e));
}

#define RFLBM_CUDA(call, what)                  \
  do {                                          \
    cudaError_t e_ = (call);                    \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Makes the handle's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int now = -1;
    if (prev >= 0 && cudaGetDevice(&now) == cudaSuccess && now != prev) cudaSetDevice(prev);
  }
};

int64_t plane_stride(int64_t n) { return (n + 63) / 64 * 64; }

// Sites one plane of a buffer holds: the box, or a z-slab's rows with its two ghost rows.
int64_t buffer_sites(const rflbm_config_t* c) {
  return (int64_t)c->nx * c->ny * (c->nz + (c->nz_global > 0 ? 2 : 0));
}

// The face exchange a z-slab needs after a step (see rflbm_slab_faces).
enum : int {
  kExchangeNone = 0,
  kExchangePull = 1,    // ping-pong: the pulled planes of the new state
  kExchangeAaFill = 2,  // AA after an even step: values the neighbours' odd step pulls
  kExchangeAaDrain = 3  // AA after an odd step: values it pushed into its ghost rows
};

int validate(const rflbm_config_t* c) {
  if (!c) return fail(RFLBM_EINVAL, "config is NULL");
  if (c->nx < 1 || c->ny < 1 || c->nz < 1)
    return fail(RFLBM_EINVAL, "box edges must be >= 1 (got %d x %d x %d)", c->nx, c->ny, c->nz);
  const int64_t n = (int64_t)c->nx * c->ny * c->nz;
  if (n >= (int64_t(1) << 31)) return fail(RFLBM_EINVAL, "box of %lld sites exceeds 2^31 - 1", (long long)n);
  if (!(c->tau > 0.5) || !std::isfinite(c->tau))
    return fail(RFLBM_EINVAL, "tau must be a finite value > 1/2 (got %g)", c->tau);
  if (!(c->kT >= 0.0) || !std::isfinite(c->kT)) return fail(RFLBM_EINVAL, "kT must be >= 0 (got %g)", c->kT);
  if (!(c->rho0 > 0.0) || !std::isfinite(c->rho0)) return fail(RFLBM_EINVAL, "rho0 must be > 0 (got %g)", c->rho0);
  if (!(c->omega_g > 0.0 && c->omega_g < 2.0))
    return fail(RFLBM_EINVAL, "omega_g must lie in (0, 2) (got %g)", c->omega_g);
  if (c->model != RFLBM_MODEL_REG && c->model != RFLBM_MODEL_BGK)
    return fail(RFLBM_EINVAL, "unknown model %d", c->model);
  if (c->storage != RFLBM_STORE_F32 && c->storage != RFLBM_STORE_F16 && c->storage != RFLBM_STORE_BF16)
    return fail(RFLBM_EINVAL, "unknown storage %d", c->storage);
  if (c->storage != RFLBM_STORE_F32 && (c->omega_g != 1.0 || c->phi_rho != RFLBM_PHI_LOCAL_RHO))
    return fail(RFLBM_EINVAL, "16-bit storage supports omega_g = 1 and the local density in Eq. 10 only");
  if (c->phi_rho != RFLBM_PHI_LOCAL_RHO && c->phi_rho != RFLBM_PHI_RHO0)
    return fail(RFLBM_EINVAL, "unknown phi_rho option %d", c->phi_rho);
  if (c->kernel < RFLBM_KERNEL_AUTO || c->kernel > RFLBM_KERNEL_TMA)
    return fail(RFLBM_EINVAL, "unknown kernel choice %d", c->kernel);
  if (c->pattern != RFLBM_PATTERN_PINGPONG && c->pattern != RFLBM_PATTERN_AA)
    return fail(RFLBM_EINVAL, "unknown streaming pattern %d", c->pattern);
  if (c->pattern == RFLBM_PATTERN_AA &&
      ((c->model == RFLBM_MODEL_REG && c->omega_g != 1.0) || c->phi_rho != RFLBM_PHI_LOCAL_RHO))
    return fail(RFLBM_EINVAL, "the AA pattern supports omega_g = 1 and the local density in Eq. 10 only");
  if (c->nz_global < 0) return fail(RFLBM_EINVAL, "nz_global must be >= 0 (got %d)", c->nz_global);
  if (c->nz_global == 0 && c->z0 != 0)
    return fail(RFLBM_EINVAL, "z0 = %d needs a z-slab (nz_global > 0)", c->z0);
  if (c->nz_global > 0) {
    if (c->z0 < 0 || (int64_t)c->z0 + c->nz > c->nz_global)
      return fail(RFLBM_EINVAL, "z-slab rows [%d, %d) outside the box of %d rows", c->z0, c->z0 + c->nz,
                  c->nz_global);
    if ((int64_t)c->nx * c->ny * c->nz_global >= (int64_t(1) << 31))
      return fail(RFLBM_EINVAL, "the decomposed box of %lld sites exceeds 2^31 - 1",
                  (long long)((int64_t)c->nx * c->ny * c->nz_global));
    if (buffer_sites(c) >= (int64_t(1) << 31))
      return fail(RFLBM_EINVAL, "the z-slab with its ghost rows exceeds 2^31 - 1 sites");
  }
  return RFLBM_OK;
}

void fill_collide_params(rflbm* h) {
  const rflbm_config_t& c = h->cfg;
  const double om = 1.0 / c.tau, og = c.omega_g;
  CollideParams& cp = h->cp;
  cp.rho0 = (float)c.rho0;
  cp.omega = (float)om;
  cp.neq_diag = (float)((1.0 - om) / bnorm(2, 0, 0));
  cp.neq_off = (float)((1.0 - om) / bnorm(1, 1, 0));
  cp.ghost_keep = (float)(1.0 - og);
  cp.sqrt_rho0 = (float)std::sqrt(c.rho0);
  // Eq. 10: phi_k = sqrt(rho kT omega_k (2 - omega_k) / (cs2 b_k)); the BGK model relaxes
  // every mode at omega (Eq. 12), Reg splits stress (omega_h) and ghost (omega_g) modes
  const double og_noise = c.model == RFLBM_MODEL_BGK ? om : og;
  cp.amp_h = (float)std::sqrt(c.kT * om * (2.0 - om));
  cp.amp_g = (float)std::sqrt(c.kT * og_noise * (2.0 - og_noise));
  h->variant.model = c.model == RFLBM_MODEL_BGK ? kModelBgk : kModelReg;
  h->variant.noise = c.kT > 0.0;
  h->variant.ghost_neq = (c.model == RFLBM_MODEL_REG) && (og != 1.0);
  h->variant.phi_rho0 = c.phi_rho == RFLBM_PHI_RHO0;
  h->variant.storage = c.storage == RFLBM_STORE_F16 ? kStoreF16 : (c.storage == RFLBM_STORE_BF16 ? kStoreBF16 : kStoreF32);
  h->elem = storage_bytes(h->variant.storage);
  // 16-bit storage: per velocity class a power of two that maps the thermal amplitude
  // sqrt(w rho0 kT / cs2) of g_i to order one (a floor of kT = 1e-6 covers kT = 0)
  const double wc[4] = {8.0 / 27.0, 2.0 / 27.0, 1.0 / 54.0, 1.0 / 216.0};
  for (int k = 0; k < 4; ++k) {
    if (h->variant.storage == kStoreF32) {
      h->ss.scale[k] = h->ss.inv_scale[k] = 1.0f;
    } else {
      const double amp = std::sqrt(3.0 * wc[k] * c.rho0 * std::max(c.kT, 1e-6));
      const int e = (int)std::lround(-std::log2(amp));
      h->ss.scale[k] = std::ldexp(1.0f, e);
      h->ss.inv_scale[k] = std::ldexp(1.0f, -e);
    }
  }
}

int ensure_staging(rflbm* h, size_t bytes) {
  if (h->staging_bytes >= bytes) return RFLBM_OK;
  if (h->staging) {
    cudaStreamSynchronize(h->stream);
    cudaFree(h->staging);
    h->staging = nullptr;
    h->staging_bytes = 0;
  }
  RFLBM_CUDA(cudaMalloc(&h->staging, bytes), "allocating the staging buffer");
  h->staging_bytes = bytes;
  return RFLBM_OK;
}

// The device-side address of a page-locked host pointer (cudaHostAlloc / cudaHostRegister
// memory, e.g. a pinned PyTorch tensor), or NULL for any other pointer. Kernels read and
// write such memory directly (over NVLink-C2C on Grace), with no staging copy.
const void* mapped_host(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free error of an unknown pointer
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int check_handle(const rflbm* h) {
  if (!h) return fail(RFLBM_EINVAL, "handle is NULL");
  return RFLBM_OK;
}

int check_ready(const rflbm* h) {
  if (int e = check_handle(h)) return e;
  if (!h->initialised) return fail(RFLBM_ESTATE, "state not initialised (call rflbm_init_rest, rflbm_init_field or rflbm_set_populations)");
  if (h->exchange != kExchangeNone)
    return fail(RFLBM_ESTATE, "the z-slab's face exchange of its last step is pending (rflbm_slab_exchange, or "
                              "rflbm_slab_faces and rflbm_slab_exchange_done)");
  return RFLBM_OK;
}

int sync(rflbm* h, const char* what) {
  RFLBM_CUDA(cudaStreamSynchronize(h->stream), what);
  int flag = 0;
  RFLBM_CUDA(cudaMemcpy(&flag, h->err, sizeof(int), cudaMemcpyDeviceToHost), "reading the error flag");
  if (flag) {
    cudaMemset(h->err, 0, sizeof(int));
    return fail(RFLBM_ETIMEOUT, "%s: a kernel gave up waiting for its bulk copies (bounded wait expired)", what);
  }
  return RFLBM_OK;
}

// The population buffer as a 4-D tensor (x, y, z, plane); box = (box_x, 1, 1, box_planes).
bool encode_map(CUtensorMap* map, void* base, const Geometry& g, uint32_t box_x, uint32_t box_planes,
                int storage) {
  return encode_population_map(map, base, g, box_x, 1, box_planes, storage);
}

// Selects the TMA step path when the box allows it and the descriptors encode.
void setup_tma(rflbm* h) {
  h->tma_width = 0;
  h->kernel = RFLBM_KERNEL_GATHER;
  const int st = h->variant.storage;
  int w = tma_segment_width(h->geo.nx);
  // rows that no width divides: ragged last segments (whose excess threads store nothing)
  if (w == 0) w = tma_ragged_width(h->geo.nx, storage_bytes(st));
  if (w == 0 || h->cfg.kernel == RFLBM_KERNEL_GATHER) return;
  const uint32_t halo = st == kStoreF32 ? 4 : 8;  // 16 bytes each side
  for (int b = 0; b < (h->aa ? 1 : 2); ++b) {
    // loads: the three planes of one source row; stores: all 27 planes of the segment
    if (!encode_map(&h->load_map[b], h->buf[b], h->geo, (uint32_t)w + 2 * halo, 3, st) ||
        !encode_map(&h->store_map[b], h->buf[b], h->geo, (uint32_t)w, kQ, st))
      return;
  }
  // AA odd form with one segment per row: three-plane stores of whole rows
  h->has_row_map = h->aa && (uint32_t)w == h->geo.nx &&
                   encode_map(&h->row_map, h->buf[0], h->geo, (uint32_t)w, 3, st);
  h->tma_width = w;
  h->kernel = RFLBM_KERNEL_TMA;
}

int64_t n_sites(const rflbm* h) { return (int64_t)h->geo.n; }

// The geometry with the view of the current state (where g_i(x) lives in buf[cur]).
Geometry vgeo(const rflbm* h) {
  Geometry g = h->geo;
  g.view = !h->aa ? kViewPull : (h->phase ? kViewFlipped : kViewNatural);
  return g;
}

}  // namespace

int rflbm_dev::record_error(int code, const char* msg, const char* detail) {
  return detail ? fail(code, "%s: %s", msg, detail) : fail(code, "%s", msg);
}

namespace {

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
  // looked up once, thread-safely (function-local static initialisation)
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return (EncodeTiledFn)p;
    return nullptr;
  }();
  return fn;
}

}  // namespace

bool rflbm_dev::encode_population_map(CUtensorMap* map, void* base, const Geometry& g, uint32_t box_x,
                                      uint32_t box_y, uint32_t box_planes, int storage) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return false;
  const cuuint64_t e = storage_bytes(storage);
  // a z-slab's buffer holds its ghost rows too
  const cuuint64_t dims[4] = {g.nx, g.ny, (cuuint64_t)g.nz + 2 * g.zlo, (cuuint64_t)kQ};
  const cuuint64_t strides[3] = {(cuuint64_t)g.nx * e, (cuuint64_t)g.nxy * e, (cuuint64_t)g.ps * e};
  const cuuint32_t box[4] = {box_x, box_y, 1, box_planes};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt = storage == kStoreF16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                 : storage == kStoreBF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                         : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(map, dt, 4, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

extern "C" {

void rflbm_config_default(rflbm_config_t* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->nx = cfg->ny = cfg->nz = 32;
  cfg->tau = 0.8;
  cfg->kT = 0.0;
  cfg->rho0 = 1.0;
  cfg->seed = 1;
  cfg->omega_g = 1.0;
  cfg->model = RFLBM_MODEL_REG;
  cfg->storage = RFLBM_STORE_F32;
  cfg->phi_rho = RFLBM_PHI_LOCAL_RHO;
  cfg->replica = 0;
  cfg->stream = nullptr;
  cfg->buffers[0] = cfg->buffers[1] = nullptr;
  cfg->device = -1;
  cfg->kernel = RFLBM_KERNEL_AUTO;
  cfg->pattern = RFLBM_PATTERN_PINGPONG;
  cfg->z0 = 0;
  cfg->nz_global = 0;
}

int64_t rflbm_config_size(void) { return (int64_t)sizeof(rflbm_config_t); }

int64_t rflbm_buffer_bytes(const rflbm_config_t* cfg) {
  if (int e = validate(cfg)) return e;
  return plane_stride(buffer_sites(cfg)) * kQ * (int64_t)(cfg->storage == RFLBM_STORE_F32 ? 4 : 2);
}

const char* rflbm_last_error(void) { return g_error.c_str(); }

rflbm_t* rflbm_create_ex(const rflbm_config_t* cfg) {
  if (validate(cfg) != RFLBM_OK) return nullptr;
  int dev = cfg->device;
  if (dev < 0) {
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
      cuda_fail(e, "querying the current device");
      return nullptr;
    }
  }
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || dev >= ndev) {
    if (e != cudaSuccess) cuda_fail(e, "querying CUDA devices");
    else fail(RFLBM_EINVAL, "device %d does not exist (%d devices)", dev, ndev);
    return nullptr;
  }
  DeviceGuard guard(dev);
  rflbm* h = new (std::nothrow) rflbm();
  if (!h) {
    fail(RFLBM_ENOMEM, "allocating the handle");
    return nullptr;
  }
  h->cfg = *cfg;
  h->device = dev;
  h->aa = cfg->pattern == RFLBM_PATTERN_AA;
  const int nbuf = h->aa ? 1 : 2;
  cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
  h->stream = (cudaStream_t)cfg->stream;
  const int64_t n = (int64_t)cfg->nx * cfg->ny * cfg->nz;
  Geometry& g = h->geo;
  g.nx = cfg->nx; g.ny = cfg->ny; g.nz = cfg->nz;
  g.nxy = (uint32_t)cfg->nx * (uint32_t)cfg->ny;
  g.n = (uint32_t)n;
  g.view = kViewPull;
  g.ps = plane_stride(buffer_sites(cfg));
  g.div_nx = make_fastdiv(g.nx);
  g.div_nxy = make_fastdiv(g.nxy);
  h->slab = cfg->nz_global > 0;
  g.zlo = h->slab ? 1u : 0u;
  g.site0 = h->slab ? g.nxy * (uint32_t)cfg->z0 : 0u;
  fill_collide_params(h);

  const size_t bytes = (size_t)g.ps * kQ * h->elem;
  if (cfg->buffers[0] || cfg->buffers[1]) {
    const bool bad = h->aa ? (!cfg->buffers[0] || cfg->buffers[1] || ((uintptr_t)cfg->buffers[0] % 256))
                           : (!cfg->buffers[0] || !cfg->buffers[1] || ((uintptr_t)cfg->buffers[0] % 256) ||
                              ((uintptr_t)cfg->buffers[1] % 256));
    if (bad) {
      fail(RFLBM_EINVAL, h->aa ? "the AA pattern takes one caller buffer (buffers[0], 256-byte aligned; buffers[1] NULL)"
                               : "caller buffers must both be given and 256-byte aligned");
      delete h;
      return nullptr;
    }
    h->buf[0] = cfg->buffers[0];
    h->buf[1] = h->aa ? nullptr : cfg->buffers[1];
    h->own_buf = false;
  } else {
    h->own_buf = true;
    for (int b = 0; b < nbuf; ++b) {
      e = cudaMalloc(&h->buf[b], bytes);
      if (e != cudaSuccess) {
        cuda_fail(e, "allocating a population buffer");
        rflbm_destroy(h);
        return nullptr;
      }
    }
  }
  // zero the buffers: the plane padding is then deterministic in state images
  for (int b = 0; b < nbuf; ++b) {
    e = cudaMemset(h->buf[b], 0, bytes);
    if (e != cudaSuccess) {
      cuda_fail(e, "clearing a population buffer");
      rflbm_destroy(h);
      return nullptr;
    }
  }
  h->stat_blocks = stats_partial_blocks(g, h->num_sms > 0 ? h->num_sms : 1);
  e = cudaMalloc((void**)&h->partials,
                 sizeof(double) * ((size_t)h->stat_blocks * kStatOutFields + 8));
  if (e == cudaSuccess) e = cudaMalloc((void**)&h->err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->err, 0, sizeof(int));
  if (e == cudaSuccess && h->slab) e = cudaEventCreateWithFlags(&h->faces_ready, cudaEventDisableTiming);
  if (e == cudaSuccess && h->slab) e = cudaEventCreateWithFlags(&h->exchanged, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    cuda_fail(e, "allocating the reduction scratch");
    rflbm_destroy(h);
    return nullptr;
  }
  setup_tma(h);
  return h;
}

rflbm_t* rflbm_create(int nx, int ny, int nz, double tau, double kT, double rho0, uint64_t seed) {
  rflbm_config_t c;
  rflbm_config_default(&c);
  c.nx = nx; c.ny = ny; c.nz = nz;
  c.tau = tau; c.kT = kT; c.rho0 = rho0; c.seed = seed;
  return rflbm_create_ex(&c);
}

void rflbm_destroy(rflbm_t* h) {
  if (!h) return;
  DeviceGuard guard(h->device);
  cudaStreamSynchronize(h->stream);
  if (h->own_buf) {
    cudaFree(h->buf[0]);
    cudaFree(h->buf[1]);
  }
  cudaFree(h->partials);
  cudaFree(h->err);
  cudaFree(h->diag_partials);
  cudaFree(h->diag_field);
  cudaFree(h->diag_spec);
  if (h->fft_ready) cufftDestroy(h->fft_plan);
  cudaFree(h->staging);
  if (h->faces_ready) cudaEventDestroy(h->faces_ready);
  if (h->exchanged) cudaEventDestroy(h->exchanged);
  if (h->halo_stream) {
    cudaStreamSynchronize(h->halo_stream);
    cudaStreamDestroy(h->halo_stream);
  }
  delete h;
}

int rflbm_init_rest(rflbm_t* h) {
  if (int e = check_handle(h)) return e;
  DeviceGuard guard(h->device);
  // the shifted rest state is all zeros
  RFLBM_CUDA(cudaMemsetAsync(h->buf[0], 0, (size_t)h->geo.ps * kQ * h->elem, h->stream),
             "clearing the populations");
  h->cur = 0;
  h->phase = 0;
  h->step = 0;
  h->exchange = kExchangeNone;
  h->initialised = true;
  return RFLBM_OK;
}

int rflbm_init_thermal(rflbm_t* h) {
  if (int e = check_handle(h)) return e;
  DeviceGuard guard(h->device);
  h->cur = 0;
  h->phase = 0;
  RFLBM_CUDA(launch_init_thermal(vgeo(h), h->cp.rho0, (float)h->cfg.kT, h->ss, h->variant.storage,
                                 (uint32_t)(h->cfg.seed & 0xffffffffu), (uint32_t)(h->cfg.seed >> 32),
                                 h->cfg.replica, h->buf[0], h->stream),
             "launching init_thermal");
  h->step = 0;
  h->exchange = kExchangeNone;
  h->initialised = true;
  return RFLBM_OK;
}

int rflbm_init_field(rflbm_t* h, const double* rho, const double* u, int on_device) {
  if (int e = check_handle(h)) return e;
  DeviceGuard guard(h->device);
  const int64_t n = n_sites(h);
  const double* drho = rho;
  const double* du = u;
  if (!on_device && (rho || u)) {
    if (int e = ensure_staging(h, sizeof(double) * 4 * n)) return e;
    double* st = (double*)h->staging;
    if (rho) {
      RFLBM_CUDA(cudaMemcpyAsync(st, rho, sizeof(double) * n, cudaMemcpyHostToDevice, h->stream), "copying rho");
      drho = st;
    }
    if (u) {
      RFLBM_CUDA(cudaMemcpyAsync(st + n, u, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, h->stream), "copying u");
      du = st + n;
    }
  }
  h->cur = 0;
  h->phase = 0;
  RFLBM_CUDA(launch_init_field(vgeo(h), h->cp.rho0, h->ss, h->variant.storage, drho, du, h->buf[0], h->stream),
             "launching init_field");
  h->step = 0;
  h->exchange = kExchangeNone;
  h->initialised = true;
  if (!on_device) return sync(h, "rflbm_init_field");
  return RFLBM_OK;
}

}  // extern "C"

namespace {

// Launches nrows rows of the handle's next step (row = y + ny z): row0 .. row0 + split - 1,
// then from row0 + split + gap on.
cudaError_t launch_rows(rflbm* h, StepParams& p, uint32_t row0, uint32_t nrows, uint32_t split = ~0u,
                        uint32_t gap = 0) {
  p.row0 = row0;
  p.nrows = nrows;
  p.row_split = split < nrows ? split : nrows;
  p.row_gap = gap;
  if (h->aa) {
    p.src = p.dst = h->buf[0];
    const bool odd = h->phase != 0;
    if (h->tma_width) {
      const TmaMaps m{&h->load_map[0], &h->store_map[0], h->tma_width, h->has_row_map ? &h->row_map : nullptr};
      return launch_step_aa_tma(m, p, h->variant, odd, h->stream);
    }
    return launch_step_aa_gather(p, h->variant, odd, h->stream);
  }
  p.src = h->buf[h->cur];
  p.dst = h->buf[1 - h->cur];
  if (h->tma_width) {
    const TmaMaps m{&h->load_map[h->cur], &h->store_map[1 - h->cur], h->tma_width};
    return launch_step_tma(m, p, h->variant, h->stream);
  }
  return launch_step_gather(p, h->variant, h->stream);
}

// One step of a z-slab: its two boundary slabs of rows first, in one launch (they write the
// faces its neighbours need), the faces-ready event, then its interior rows, which run while
// the faces move.
cudaError_t slab_step(rflbm* h, StepParams& p) {
  const uint32_t ny = h->geo.ny, nz = h->geo.nz;
  cudaError_t e = nz <= 2 ? launch_rows(h, p, 0, ny * nz) : launch_rows(h, p, 0, 2 * ny, ny, (nz - 2) * ny);
  if (e == cudaSuccess) e = cudaEventRecord(h->faces_ready, h->stream);
  if (e == cudaSuccess && nz > 2) e = launch_rows(h, p, ny, (nz - 2) * ny);
  return e;
}

}  // namespace

extern "C" {

int rflbm_step(rflbm_t* h, int64_t n) {
  if (int e = check_ready(h)) return e;
  if (n < 0) return fail(RFLBM_EINVAL, "negative step count %lld", (long long)n);
  if (h->slab && n > 1)
    return fail(RFLBM_EINVAL, "a z-slab takes one step per call (its faces are exchanged between steps)");
  DeviceGuard guard(h->device);
  StepParams p;
  p.geo = h->geo;
  p.cp = h->cp;
  p.ss = h->ss;
  p.key0 = (uint32_t)(h->cfg.seed & 0xffffffffu);
  p.key1 = (uint32_t)(h->cfg.seed >> 32);
  p.rk = philox_round_keys(p.key0, p.key1);
  p.replica = h->cfg.replica;
  p.err = h->err;
  p.test_extra_tx = h->test_extra_tx;
  for (int64_t t = 0; t < n; ++t) {
    p.step = (uint32_t)h->step;
    const cudaError_t e = h->slab ? slab_step(h, p) : launch_rows(h, p, 0, h->geo.ny * h->geo.nz);
    if (e != cudaSuccess) return cuda_fail(e, "launching the step kernel");
    if (h->slab) h->exchange = !h->aa ? kExchangePull : (h->phase ? kExchangeAaDrain : kExchangeAaFill);
    if (h->aa) h->phase ^= 1;
    else h->cur = 1 - h->cur;
    ++h->step;
  }
  return RFLBM_OK;
}

int rflbm_moments(rflbm_t* h, double* rho, double* u, double* pi, int on_device) {
  if (int e = check_ready(h)) return e;
  DeviceGuard guard(h->device);
  const int64_t n = n_sites(h);
  double *drho = rho, *du = u, *dpi = pi;
  if (!on_device) {
    if (int e = ensure_staging(h, sizeof(double) * 10 * n)) return e;
    double* st = (double*)h->staging;
    drho = rho ? st : nullptr;
    du = u ? st + n : nullptr;
    dpi = pi ? st + 4 * n : nullptr;
  }
  RFLBM_CUDA(launch_moments(vgeo(h), h->cp.rho0, h->ss, h->variant.storage, h->buf[h->cur], drho, du, dpi, h->stream),
             "launching moments");
  if (!on_device) {
    if (rho) RFLBM_CUDA(cudaMemcpyAsync(rho, drho, sizeof(double) * n, cudaMemcpyDeviceToHost, h->stream), "copying rho");
    if (u) RFLBM_CUDA(cudaMemcpyAsync(u, du, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, h->stream), "copying u");
    if (pi) RFLBM_CUDA(cudaMemcpyAsync(pi, dpi, sizeof(double) * 6 * n, cudaMemcpyDeviceToHost, h->stream), "copying pi");
  }
  return sync(h, "rflbm_moments");
}

int rflbm_stats(rflbm_t* h, rflbm_stats_t* out) {
  if (int e = check_ready(h)) return e;
  if (!out) return fail(RFLBM_EINVAL, "stats output is NULL");
  DeviceGuard guard(h->device);
  double* res = h->partials + (size_t)h->stat_blocks * kStatOutFields;
  RFLBM_CUDA(launch_stats(vgeo(h), h->cp.rho0, h->ss, h->variant.storage, h->buf[h->cur], h->partials,
                          h->stat_blocks, res, h->stream),
             "launching stats");
  double host[kStatOutFields];
  RFLBM_CUDA(cudaMemcpyAsync(host, res, sizeof(host), cudaMemcpyDeviceToHost, h->stream), "copying stats");
  if (int e = sync(h, "rflbm_stats")) return e;
  out->step = h->step;
  out->mass = (double)n_sites(h) * h->cfg.rho0 + host[0];
  out->momentum[0] = host[1];
  out->momentum[1] = host[2];
  out->momentum[2] = host[3];
  out->max_speed = host[4];
  out->nonfinite = (int64_t)host[5];
  if (out->nonfinite > 0)
    return fail(RFLBM_EUNSTABLE, "%lld sites are unstable (non-finite values or non-positive density) at step %lld",
                (long long)out->nonfinite, (long long)h->step);
  return RFLBM_OK;
}

static int get_pops(rflbm_t* h, void* f, int on_device, bool f64) {
  if (int e = check_ready(h)) return e;
  if (!f) return fail(RFLBM_EINVAL, "output is NULL");
  DeviceGuard guard(h->device);
  const int64_t n = n_sites(h);
  const size_t bytes = (size_t)kQ * n * (f64 ? sizeof(double) : sizeof(float));
  void* dst = f;
  bool copy_back = false;
  if (!on_device) {
    dst = const_cast<void*>(mapped_host(f));
    if (!dst) {
      if (int e = ensure_staging(h, bytes)) return e;
      dst = h->staging;
      copy_back = true;
    }
  }
  const int st = h->variant.storage;
  const Geometry g = vgeo(h);
  cudaError_t e = f64 ? launch_get_populations_f64(g, h->cp.rho0, h->ss, st, h->buf[h->cur], (double*)dst, h->stream)
                      : launch_get_populations_f32(g, h->cp.rho0, h->ss, st, h->buf[h->cur], (float*)dst, h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching get_populations");
  if (copy_back) RFLBM_CUDA(cudaMemcpyAsync(f, dst, bytes, cudaMemcpyDeviceToHost, h->stream), "copying populations");
  return sync(h, "rflbm_get_populations");
}

static int set_pops(rflbm_t* h, const void* f, int on_device, bool f64) {
  if (int e = check_handle(h)) return e;
  if (!f) return fail(RFLBM_EINVAL, "input is NULL");
  DeviceGuard guard(h->device);
  const int64_t n = n_sites(h);
  const size_t bytes = (size_t)kQ * n * (f64 ? sizeof(double) : sizeof(float));
  const void* src = f;
  if (!on_device) {
    src = mapped_host(f);
    if (!src) {
      if (int e = ensure_staging(h, bytes)) return e;
      RFLBM_CUDA(cudaMemcpyAsync(h->staging, f, bytes, cudaMemcpyHostToDevice, h->stream), "copying populations");
      src = h->staging;
    }
  }
  // the state after this call is step h->step, held in buffer 0 (AA: natural view)
  h->cur = 0;
  h->phase = 0;
  const int st = h->variant.storage;
  const Geometry g = vgeo(h);
  cudaError_t e = f64 ? launch_set_populations_f64(g, h->cp.rho0, h->ss, st, (const double*)src, h->buf[0], h->stream)
                      : launch_set_populations_f32(g, h->cp.rho0, h->ss, st, (const float*)src, h->buf[0], h->stream);
  if (e != cudaSuccess) return cuda_fail(e, "launching set_populations");
  h->exchange = kExchangeNone;
  h->initialised = true;
  if (!on_device) return sync(h, "rflbm_set_populations");
  return RFLBM_OK;
}

int rflbm_get_populations(rflbm_t* h, double* f, int on_device) { return get_pops(h, f, on_device, true); }
int rflbm_get_populations_f32(rflbm_t* h, float* f, int on_device) { return get_pops(h, f, on_device, false); }
int rflbm_set_populations(rflbm_t* h, const double* f, int on_device) { return set_pops(h, f, on_device, true); }
int rflbm_set_populations_f32(rflbm_t* h, const float* f, int on_device) { return set_pops(h, f, on_device, false); }

int rflbm_get_sites(rflbm_t* h, const int64_t* sites, int64_t n, double* f) {
  if (int e = check_ready(h)) return e;
  if (n < 0 || (n > 0 && (!sites || !f))) return fail(RFLBM_EINVAL, "invalid site list");
  if (n == 0) return RFLBM_OK;
  for (int64_t j = 0; j < n; ++j)
    if (sites[j] < 0 || sites[j] >= n_sites(h))
      return fail(RFLBM_EINVAL, "site index %lld out of range [0, %lld)", (long long)sites[j], (long long)n_sites(h));
  DeviceGuard guard(h->device);
  const size_t bytes_sites = sizeof(int64_t) * n, bytes_out = sizeof(double) * kQ * n;
  if (int e = ensure_staging(h, bytes_sites + bytes_out)) return e;
  int64_t* dsites = (int64_t*)h->staging;
  double* dout = (double*)((char*)h->staging + bytes_sites);
  RFLBM_CUDA(cudaMemcpyAsync(dsites, sites, bytes_sites, cudaMemcpyHostToDevice, h->stream), "copying sites");
  RFLBM_CUDA(launch_get_sites(vgeo(h), h->cp.rho0, h->ss, h->variant.storage, h->buf[h->cur], dsites, n, dout, h->stream),
             "launching get_sites");
  RFLBM_CUDA(cudaMemcpyAsync(f, dout, bytes_out, cudaMemcpyDeviceToHost, h->stream), "copying site populations");
  return sync(h, "rflbm_get_sites");
}

static int ensure_diag_partials(rflbm* h, size_t bytes) {
  if (h->diag_partials_bytes >= bytes) return RFLBM_OK;
  cudaStreamSynchronize(h->stream);
  cudaFree(h->diag_partials);
  h->diag_partials = nullptr;
  h->diag_partials_bytes = 0;
  RFLBM_CUDA(cudaMalloc((void**)&h->diag_partials, bytes), "allocating diagnostics scratch");
  h->diag_partials_bytes = bytes;
  return RFLBM_OK;
}

int rflbm_mode_sums(rflbm_t* h, double* sum, double* sumsq) {
  if (int e = check_ready(h)) return e;
  if (!sum || !sumsq) return fail(RFLBM_EINVAL, "outputs are NULL");
  DeviceGuard guard(h->device);
  const int64_t rows = mode_sum_blocks(h->geo);
  if (int e = ensure_diag_partials(h, sizeof(double) * (size_t)(rows + 1) * 2 * kQ)) return e;
  double* out = h->diag_partials + rows * 2 * kQ;
  RFLBM_CUDA(launch_mode_sums(vgeo(h), h->ss, h->variant.storage, h->buf[h->cur], h->diag_partials, out, h->stream),
             "launching mode sums");
  double host[2 * kQ];
  RFLBM_CUDA(cudaMemcpyAsync(host, out, sizeof(host), cudaMemcpyDeviceToHost, h->stream), "copying mode sums");
  if (int e = sync(h, "rflbm_mode_sums")) return e;
  for (int k = 0; k < kQ; ++k) {
    sum[k] = host[k];
    sumsq[k] = host[kQ + k];
  }
  return RFLBM_OK;
}

int rflbm_shell_count(const rflbm_t* h) {
  if (int e = check_handle(h)) return e;
  const double L = (double)std::max(h->geo.nx, std::max(h->geo.ny, h->geo.nz));
  return (int)std::llround(L * std::sqrt(3.0) / 2.0) + 1;
}

int rflbm_structure_factor(rflbm_t* h, int field, int nshell, double* s_sum, double* count) {
  if (int e = check_ready(h)) return e;
  if (field < RFLBM_FIELD_RHO || field > RFLBM_FIELD_PYZ) return fail(RFLBM_EINVAL, "unknown field %d", field);
  if (nshell < 1 || nshell > 3072) return fail(RFLBM_EINVAL, "nshell must lie in [1, 3072] (got %d)", nshell);
  if (!s_sum || !count) return fail(RFLBM_EINVAL, "outputs are NULL");
  if (h->slab) return fail(RFLBM_ESTATE, "the structure factor needs the whole box, not one z-slab of it");
  DeviceGuard guard(h->device);
  const Geometry& g = h->geo;
  const size_t nspec = (size_t)g.nz * g.ny * (g.nx / 2 + 1);
  if (!h->fft_ready) {
    RFLBM_CUDA(cudaMalloc((void**)&h->diag_field, sizeof(double) * g.n), "allocating the field buffer");
    RFLBM_CUDA(cudaMalloc(&h->diag_spec, sizeof(cufftDoubleComplex) * nspec), "allocating the spectrum");
    if (cufftPlan3d(&h->fft_plan, (int)g.nz, (int)g.ny, (int)g.nx, CUFFT_D2Z) != CUFFT_SUCCESS)
      return fail(RFLBM_ECUDA, "cufftPlan3d failed for %u x %u x %u", g.nx, g.ny, g.nz);
    h->fft_ready = true;
  }
  if (cufftSetStream(h->fft_plan, h->stream) != CUFFT_SUCCESS) return fail(RFLBM_ECUDA, "cufftSetStream failed");
  const int blocks = std::max(1, std::min(4 * std::max(h->num_sms, 1), (int)((nspec + 255) / 256)));
  if (int e = ensure_diag_partials(h, sizeof(double) * (size_t)(blocks + 1) * 2 * nshell)) return e;
  double* out = h->diag_partials + (size_t)blocks * 2 * nshell;
  RFLBM_CUDA(launch_field(vgeo(h), h->ss, h->variant.storage, h->buf[h->cur], field, h->diag_field, h->stream),
             "launching the field kernel");
  if (cufftExecD2Z(h->fft_plan, h->diag_field, (cufftDoubleComplex*)h->diag_spec) != CUFFT_SUCCESS)
    return fail(RFLBM_ECUDA, "cufftExecD2Z failed");
  RFLBM_CUDA(launch_shell_bins(g, h->diag_spec, nshell, blocks, h->diag_partials, out, h->stream),
             "launching the shell binning");
  std::vector<double> host((size_t)2 * nshell);
  RFLBM_CUDA(cudaMemcpyAsync(host.data(), out, sizeof(double) * host.size(), cudaMemcpyDeviceToHost, h->stream),
             "copying the shell sums");
  if (int e = sync(h, "rflbm_structure_factor")) return e;
  for (int n = 0; n < nshell; ++n) {
    s_sum[n] = host[n];
    count[n] = host[nshell + n];
  }
  return RFLBM_OK;
}

int64_t rflbm_state_bytes(const rflbm_t* h) {
  if (int e = check_handle(h)) return e;
  return h->geo.ps * kQ * (int64_t)h->elem;
}

int rflbm_save_state(rflbm_t* h, void* image, int on_device) {
  if (int e = check_ready(h)) return e;
  if (!image) return fail(RFLBM_EINVAL, "image is NULL");
  if (h->slab && h->aa)
    return fail(RFLBM_ESTATE, "state images of z-slabs are supported in the ping-pong pattern only");
  DeviceGuard guard(h->device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (!h->aa) {
    RFLBM_CUDA(cudaMemcpyAsync(image, h->buf[h->cur], (size_t)rflbm_state_bytes(h), kind, h->stream),
               "copying the state image");
    return sync(h, "rflbm_save_state");
  }
  // AA: the image is the pull layout. Flipped view: image plane q = buffer plane 26 - q.
  // Natural view: image plane P(i) at y = buffer plane P(i) at y + c_i (one shifted copy
  // per plane through a one-plane scratch buffer).
  const size_t plane_bytes = (size_t)h->geo.ps * h->elem;
  char* const img = static_cast<char*>(image);
  const char* const buf = static_cast<const char*>(h->buf[0]);
  if (!h->phase) {
    if (int e = ensure_staging(h, plane_bytes)) return e;
  }
  for (int i = 0; i < kQ; ++i) {
    const int q = plane_of(i);
    if (h->phase) {
      RFLBM_CUDA(cudaMemcpyAsync(img + q * plane_bytes, buf + (kQ - 1 - q) * plane_bytes, plane_bytes, kind, h->stream),
                 "copying a state image plane");
      continue;
    }
    void* out = on_device ? (void*)(img + q * plane_bytes) : h->staging;
    RFLBM_CUDA(launch_image_plane(h->geo, h->elem, buf + q * plane_bytes, cx_of(i), cy_of(i), cz_of(i), out, h->stream),
               "launching the image plane kernel");
    if (!on_device)
      RFLBM_CUDA(cudaMemcpyAsync(img + q * plane_bytes, h->staging, plane_bytes, cudaMemcpyDeviceToHost, h->stream),
                 "copying a state image plane");
  }
  return sync(h, "rflbm_save_state");
}

int rflbm_load_state(rflbm_t* h, const void* image, int on_device) {
  if (int e = check_handle(h)) return e;
  if (!image) return fail(RFLBM_EINVAL, "image is NULL");
  if (h->slab && h->aa)
    return fail(RFLBM_ESTATE, "state images of z-slabs are supported in the ping-pong pattern only");
  DeviceGuard guard(h->device);
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (!h->aa) {
    RFLBM_CUDA(cudaMemcpyAsync(h->buf[0], image, (size_t)rflbm_state_bytes(h), kind, h->stream),
               "copying the state image");
  } else {
    // AA: the pull-layout image becomes the flipped view (buffer plane 26 - q = image plane q)
    const size_t plane_bytes = (size_t)h->geo.ps * h->elem;
    const char* const img = static_cast<const char*>(image);
    char* const buf = static_cast<char*>(h->buf[0]);
    for (int q = 0; q < kQ; ++q)
      RFLBM_CUDA(cudaMemcpyAsync(buf + (kQ - 1 - q) * plane_bytes, img + q * plane_bytes, plane_bytes, kind, h->stream),
                 "copying a state image plane");
    h->phase = 1;
  }
  h->cur = 0;
  h->exchange = kExchangeNone;
  h->initialised = true;
  return sync(h, "rflbm_load_state");
}

int64_t rflbm_get_step(const rflbm_t* h) {
  if (check_handle(h)) return RFLBM_EINVAL;
  return h->step;
}

int rflbm_set_step(rflbm_t* h, int64_t step) {
  if (int e = check_handle(h)) return e;
  if (step < 0) return fail(RFLBM_EINVAL, "negative step %lld", (long long)step);
  h->step = step;
  return RFLBM_OK;
}

int rflbm_set_stream(rflbm_t* h, void* stream) {
  if (int e = check_handle(h)) return e;
  h->stream = (cudaStream_t)stream;
  h->cfg.stream = stream;
  return RFLBM_OK;
}

int rflbm_synchronize(rflbm_t* h) {
  if (int e = check_handle(h)) return e;
  DeviceGuard guard(h->device);
  return sync(h, "rflbm_synchronize");
}

int rflbm_get_dims(const rflbm_t* h, int* nx, int* ny, int* nz) {
  if (int e = check_handle(h)) return e;
  if (nx) *nx = h->cfg.nx;
  if (ny) *ny = h->cfg.ny;
  if (nz) *nz = h->cfg.nz;
  return RFLBM_OK;
}

int rflbm_launches_per_step(const rflbm_t* h) {
  if (int e = check_handle(h)) return e;
  if (!h->slab) return 1;
  return h->geo.nz <= 2 ? 1 : 2;  // a z-slab: boundary rows, interior rows
}

int rflbm_step_path(const rflbm_t* h, int* width) {
  if (int e = check_handle(h)) return e;
  if (width) *width = h->tma_width;
  return h->kernel;
}

int rflbm_step_sites_per_thread(const rflbm_t* h) {
  if (int e = check_handle(h)) return e;
  if (h->kernel != RFLBM_KERNEL_TMA) return 1;
  if (h->aa) return aa_uses_pairs(h->variant, h->phase != 0, h->has_row_map) ? 2 : 1;
  return tma_uses_pairs(h->variant) ? 2 : 1;
}

}  // extern "C"

namespace {

// One face of a z-slab's buffer: the 9 planes of the populations with c_z = cz at buffer
// row zb, as three runs of three adjacent planes (internal plane order: run b holds the
// planes 3 (3 b + cz + 1) + (0, 1, 2), i.e. c_y = b - 1 and c_x = -1, 0, +1).
rflbm_face_t face_of(const rflbm* h, void* buffer, uint32_t zb, int cz) {
  rflbm_face_t f;
  const int64_t pitch = h->geo.ps * (int64_t)h->elem;
  for (int b = 0; b < 3; ++b) {
    const int plane = 3 * (3 * b + cz + 1);
    f.run[b] = static_cast<char*>(buffer) + plane * pitch + (int64_t)zb * h->geo.nxy * (int64_t)h->elem;
  }
  f.plane_pitch = pitch;
  f.row_bytes = (int64_t)h->geo.nxy * (int64_t)h->elem;
  return f;
}

// Largest plane pitch (bytes) for which rflbm_slab_exchange moves a face as one 3-D copy,
// when set below the device's maximum copy pitch by rflbm_testing_slab_copy_pitch_limit (0:
// the device's).
int64_t g_face_copy_pitch_limit = 0;

// Moves one face: as one 3-D copy (3 runs, 9 planes apart, of 3 plane rows) when both faces
// have that shape and their plane pitch is within the copy pitch limit (measured on one
// 128^3 slab periodic through its own faces: 78 us per step against 94 us with one 2-D copy
// per run), else one copy per plane row.
cudaError_t copy_face(const rflbm_face_t& from, const rflbm_face_t& to, int device, cudaStream_t hs) {
  int max_pitch = 0;
  if (cudaError_t e = cudaDeviceGetAttribute(&max_pitch, cudaDevAttrMaxPitch, device)) return e;
  int64_t limit = max_pitch;
  if (g_face_copy_pitch_limit > 0 && g_face_copy_pitch_limit < limit) limit = g_face_copy_pitch_limit;
  bool runs9 = from.plane_pitch <= limit && to.plane_pitch <= limit;
  for (int b = 1; b < 3; ++b) {
    runs9 = runs9 && static_cast<char*>(from.run[b]) - static_cast<char*>(from.run[0]) == 9 * b * from.plane_pitch;
    runs9 = runs9 && static_cast<char*>(to.run[b]) - static_cast<char*>(to.run[0]) == 9 * b * to.plane_pitch;
  }
  if (runs9) {
    cudaMemcpy3DParms m = {};
    m.srcPtr = make_cudaPitchedPtr(from.run[0], (size_t)from.plane_pitch, (size_t)from.row_bytes, 9);
    m.dstPtr = make_cudaPitchedPtr(to.run[0], (size_t)to.plane_pitch, (size_t)to.row_bytes, 9);
    m.extent = make_cudaExtent((size_t)from.row_bytes, 3, 3);
    m.kind = cudaMemcpyDeviceToDevice;
    return cudaMemcpy3DAsync(&m, hs);
  }
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a)
      if (cudaError_t e = cudaMemcpyAsync(static_cast<char*>(to.run[b]) + a * to.plane_pitch,
                                          static_cast<const char*>(from.run[b]) + a * from.plane_pitch,
                                          (size_t)from.row_bytes, cudaMemcpyDeviceToDevice, hs))
        return e;
  return cudaSuccess;
}

int check_slab(const rflbm* h) {
  if (int e = check_handle(h)) return e;
  if (!h->slab) return fail(RFLBM_EINVAL, "not a z-slab handle (nz_global = 0)");
  return RFLBM_OK;
}

}  // namespace

extern "C" {

int rflbm_slab_faces(rflbm_t* h, rflbm_face_t* send_up, rflbm_face_t* send_down, rflbm_face_t* recv_below,
                     rflbm_face_t* recv_above) {
  if (int e = check_slab(h)) return e;
  if (h->exchange == kExchangeNone) return fail(RFLBM_ESTATE, "no face exchange is pending");
  const uint32_t nz = h->geo.nz;
  void* const buf = h->aa ? h->buf[0] : h->buf[h->cur];
  // buffer rows: 0 ghost below, 1 .. nz own rows, nz + 1 ghost above
  rflbm_face_t f[4];
  switch (h->exchange) {
    case kExchangePull:  // the new state's populations that cross a face, pulled next step
      f[0] = face_of(h, buf, nz, +1); f[1] = face_of(h, buf, 1, -1);
      f[2] = face_of(h, buf, 0, +1);  f[3] = face_of(h, buf, nz + 1, -1);
      break;
    case kExchangeAaFill:  // an even AA step left them in the slots of the opposite direction
      f[0] = face_of(h, buf, nz, -1); f[1] = face_of(h, buf, 1, +1);
      f[2] = face_of(h, buf, 0, -1);  f[3] = face_of(h, buf, nz + 1, +1);
      break;
    default:  // an odd AA step pushed them into the ghost rows; they return to their owners
      f[0] = face_of(h, buf, nz + 1, +1); f[1] = face_of(h, buf, 0, -1);
      f[2] = face_of(h, buf, 1, +1);      f[3] = face_of(h, buf, nz, -1);
      break;
  }
  if (send_up) *send_up = f[0];
  if (send_down) *send_down = f[1];
  if (recv_below) *recv_below = f[2];
  if (recv_above) *recv_above = f[3];
  return RFLBM_OK;
}

int rflbm_slab_faces_ready(rflbm_t* h, void* stream) {
  if (int e = check_slab(h)) return e;
  if (h->exchange == kExchangeNone) return fail(RFLBM_ESTATE, "no face exchange is pending");
  DeviceGuard guard(h->device);
  RFLBM_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, h->faces_ready, 0), "waiting for the faces");
  return RFLBM_OK;
}

int rflbm_slab_exchange_done(rflbm_t* h, void* stream) {
  if (int e = check_slab(h)) return e;
  if (h->exchange == kExchangeNone) return fail(RFLBM_ESTATE, "no face exchange is pending");
  DeviceGuard guard(h->device);
  RFLBM_CUDA(cudaEventRecord(h->exchanged, (cudaStream_t)stream), "recording the end of the exchange");
  RFLBM_CUDA(cudaStreamWaitEvent(h->stream, h->exchanged, 0), "ordering the next step after the exchange");
  h->exchange = kExchangeNone;
  return RFLBM_OK;
}

int rflbm_slab_exchange(rflbm_t* const* slabs, int n) {
  if (!slabs || n < 1) return fail(RFLBM_EINVAL, "no slabs given");
  for (int k = 0; k < n; ++k) {
    if (int e = check_slab(slabs[k])) return e;
    const rflbm* a = slabs[k];
    const rflbm* b = slabs[0];
    if (a->exchange == kExchangeNone) return fail(RFLBM_ESTATE, "slab %d has no face exchange pending", k);
    if (a->exchange != b->exchange || a->device != b->device || a->geo.nx != b->geo.nx || a->geo.ny != b->geo.ny ||
        a->elem != b->elem || a->aa != b->aa || a->cfg.nz_global != b->cfg.nz_global)
      return fail(RFLBM_EINVAL, "slab %d does not match slab 0 (device, row shape, storage, pattern or step)", k);
    const int up = (k + 1) % n;
    if ((slabs[up]->cfg.z0 - (a->cfg.z0 + a->cfg.nz)) % a->cfg.nz_global != 0)
      return fail(RFLBM_EINVAL, "slab %d is not followed by its upper neighbour (slabs must be given in z order)", k);
  }
  rflbm* h0 = slabs[0];
  DeviceGuard guard(h0->device);
  if (!h0->halo_stream)
    RFLBM_CUDA(cudaStreamCreateWithFlags(&h0->halo_stream, cudaStreamNonBlocking), "creating the halo stream");
  cudaStream_t hs = h0->halo_stream;
  // the copies start once every slab's boundary rows are written (which also means that
  // its previous step, the last reader of the rows the copies overwrite, is complete)
  for (int k = 0; k < n; ++k)
    RFLBM_CUDA(cudaStreamWaitEvent(hs, slabs[k]->faces_ready, 0), "waiting for the faces");
  for (int k = 0; k < n; ++k) {
    rflbm_face_t up_k, down_k, below_k, above_k, up_u, down_u, below_u, above_u;
    rflbm* lo = slabs[k];
    rflbm* hi = slabs[(k + 1) % n];
    rflbm_slab_faces(lo, &up_k, &down_k, &below_k, &above_k);
    rflbm_slab_faces(hi, &up_u, &down_u, &below_u, &above_u);
    // the lower slab's upward face into the upper slab's row below it, and back down
    RFLBM_CUDA(copy_face(up_k, below_u, h0->device, hs), "copying a face up");
    RFLBM_CUDA(copy_face(down_u, above_k, h0->device, hs), "copying a face down");
  }
  for (int k = 0; k < n; ++k)
    if (int e = rflbm_slab_exchange_done(slabs[k], hs)) return e;
  return RFLBM_OK;
}

int rflbm_testing_slab_copy_pitch_limit(int64_t bytes) {
  if (bytes < 0) return fail(RFLBM_EINVAL, "negative pitch limit");
  g_face_copy_pitch_limit = bytes;
  return RFLBM_OK;
}

int rflbm_testing_expect_extra_bytes(rflbm_t* h, uint32_t bytes) {
  if (int e = check_handle(h)) return e;
  if (bytes > (1u << 20)) return fail(RFLBM_EINVAL, "extra byte count %u above 2^20", bytes);
  h->test_extra_tx = bytes;
  return RFLBM_OK;
}

int rflbm_philox4x32_10(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out, int64_t n) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return fail(RFLBM_EINVAL, "invalid arguments");
  if (n == 0) return RFLBM_OK;
  uint32_t *dctr = nullptr, *dout = nullptr;
  const size_t bytes = sizeof(uint32_t) * 4 * n;
  RFLBM_CUDA(cudaMalloc(&dctr, bytes), "allocating counters");
  cudaError_t e = cudaMalloc(&dout, bytes);
  if (e == cudaSuccess) e = cudaMemcpy(dctr, ctr, bytes, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_philox(dctr, k0, k1, dout, n, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, bytes, cudaMemcpyDeviceToHost);
  cudaFree(dctr);
  cudaFree(dout);
  if (e != cudaSuccess) return cuda_fail(e, "rflbm_philox4x32_10");
  return RFLBM_OK;
}

int rflbm_site_normals(uint64_t seed, int64_t step, uint32_t replica, const uint32_t* sites,
                       int64_t n, float* out) {
  if (n < 0 || (n > 0 && (!sites || !out)) || step < 0) return fail(RFLBM_EINVAL, "invalid arguments");
  if (n == 0) return RFLBM_OK;
  uint32_t* ds = nullptr;
  float* dout = nullptr;
  RFLBM_CUDA(cudaMalloc(&ds, sizeof(uint32_t) * n), "allocating sites");
  cudaError_t e = cudaMalloc(&dout, sizeof(float) * 24 * n);
  if (e == cudaSuccess) e = cudaMemcpy(ds, sites, sizeof(uint32_t) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = launch_site_normals((uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32), (uint32_t)step,
                            replica, ds, n, dout, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(out, dout, sizeof(float) * 24 * n, cudaMemcpyDeviceToHost);
  cudaFree(ds);
  cudaFree(dout);
  if (e != cudaSuccess) return cuda_fail(e, "rflbm_site_normals");
  return RFLBM_OK;
}

}  // extern "C"
