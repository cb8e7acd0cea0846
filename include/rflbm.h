/*
 * rflbm.h - C ABI of a GB300 (sm_103a) implementation of the regularized fluctuating
 * lattice Boltzmann model on the D3Q27 lattice (Reg-FLBM; Lauricella, Montessori,
 * Tiribocchi, Succi, arXiv 2507.08820).
 *
 * One handle holds one periodic box of nx*ny*nz lattice sites and advances it with the
 * fused per-site stream-and-collide step of Eq. 25 (Sec. II.B): density, velocity and
 * the second Hermite moment are projected from the 27 populations, the equilibrium is
 * the full D3Q27 Hermite expansion of Eq. 26 with the recursive coefficients of Eq. 21,
 * the stress modes relax at omega_h = 1/tau, the ghost modes at omega_g (1 in the
 * paper), Gaussian noise with the amplitude of Eq. 10 enters every non-conserved mode
 * (k = 4..26 of Table II), the populations are rebuilt by the back transform of Eq. 11
 * and streamed (Eq. 8).
 *
 * Conventions used by every entry point
 *   - Sites: s = x + nx*(y + ny*z), x fastest; every field is indexed by s.
 *   - Populations: 27 planes of N = nx*ny*nz values, plane i holding f_i for every site
 *     ("structure of arrays", element [i*N + s]). Velocity order (Table I groups; order
 *     inside a group as follows): i = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z; 7..18 = the
 *     (x,y), (x,z), (y,z) diagonals each as (+,+),(+,-),(-,+),(-,-); 19..26 =
 *     (+-1,+-1,+-1) counting in binary with x slowest and + before -.
 *   - Time: the state held is the pre-collision f(x, t) of step t (t = 0 after an init
 *     call). rflbm_step(h, n) takes steps t .. t+n-1; the noise of step t at site s is
 *     drawn from Philox4x32-10 (Salmon et al., SC'11) at counter (s, t, j, replica),
 *     j = 0..5, key (seed mod 2^32, seed div 2^32), Box-Muller on word pairs (0,1) and
 *     (2,3), uniforms (x + 1/2) 2^-32, r_k = n[k - 4].
 *   - on_device: 0 = the pointer is host memory (pinned or pageable), 1 = CUDA device
 *     memory of the handle's device. The caller owns every buffer it passes; the
 *     library never frees caller memory.
 *   - Errors: functions returning int return RFLBM_OK (0) or a negative rflbm_status;
 *     functions returning a pointer return NULL. rflbm_last_error() then describes the
 *     failure (thread-local, valid until the next call on the same thread). Work is
 *     enqueued on the handle's stream; a CUDA error raised by a kernel surfaces at the
 *     next call that synchronises (moments, stats, get_*, synchronize).
 *   - Threads: different handles may be used from different threads at once; one handle
 *     must not be used by two threads at the same time (its calls share the handle's
 *     stream, state counters and scratch buffers).
 */
#ifndef RFLBM_H
#define RFLBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rflbm rflbm_t;

typedef enum {
  RFLBM_OK = 0,
  RFLBM_EINVAL = -1,     /* invalid argument (sizes, tau <= 1/2, kT < 0, rho0 <= 0, ...) */
  RFLBM_ENOMEM = -2,     /* device or host allocation failed */
  RFLBM_ECUDA = -3,      /* CUDA runtime error (no device, launch or kernel failure) */
  RFLBM_EUNSTABLE = -4,  /* the state holds non-finite values or non-positive densities
                            (reported by rflbm_stats) */
  RFLBM_ETIMEOUT = -5,   /* a bounded device wait expired */
  RFLBM_ESTATE = -6      /* call not valid in the handle's current state */
} rflbm_status;

typedef enum {
  RFLBM_MODEL_REG = 0,   /* Reg-FLBM, Eq. 25 (Eq. 24 split with omega_g) */
  RFLBM_MODEL_BGK = 1    /* BGK-FLBM, Eq. 12 with the equilibrium of Eq. 26 (Sec. III) */
} rflbm_model;

/* Population storage. All formats hold g_i = f_i - w_i rho0 (the rest state is 0) and all
 * arithmetic is float32. The 16-bit formats halve the bytes per site update (108 instead
 * of 216); they store g_i * 2^e with one power of two per velocity class |c_i|^2 chosen so
 * that the thermal amplitude sqrt(w_i rho0 max(kT, 1e-6) / cs2) is of order one, and they
 * support the paper's configuration (omega_g = 1, local rho in Eq. 10) only. */
typedef enum {
  RFLBM_STORE_F32 = 0,   /* float32 */
  RFLBM_STORE_F16 = 1,   /* IEEE float16 (11-bit significand) */
  RFLBM_STORE_BF16 = 2   /* bfloat16 (8-bit significand) */
} rflbm_storage;

typedef enum {
  RFLBM_PHI_LOCAL_RHO = 0, /* rho in Eq. 10 is the site's density (default) */
  RFLBM_PHI_RHO0 = 1       /* rho in Eq. 10 is the reference density rho0 */
} rflbm_phi_rho;

/* Step kernels. Both compute the same step; they differ in how the 27 neighbours are
 * fetched. The TMA kernel runs in row segments of 128, 192, 96, 64 or 32 sites: the first
 * that divides nx when nx is a multiple of 32; otherwise, when a row is a whole number of
 * 16-byte units (nx a multiple of 4 in float32, of 8 in 16-bit storage), the width whose
 * segments cover the row with the fewest idle threads per measured efficiency, the last
 * segment of each row ending past it, provided at least 77 % of the threads stay busy
 * (rflbm_step_path reports the width). On other boxes every choice runs the general kernel.
 * Some variants of the TMA kernel update two sites per thread with packed arithmetic
 * (rflbm_step_sites_per_thread), bit for bit like the one-site forms. */
typedef enum {
  RFLBM_KERNEL_AUTO = 0,    /* TMA when the box allows it, else the general kernel */
  RFLBM_KERNEL_GATHER = 1,  /* one thread per site, 27 addressed loads */
  RFLBM_KERNEL_TMA = 2      /* one CTA per row segment, TMA tensor loads and stores */
} rflbm_kernel;

/* Streaming pattern (Eq. 8 carried out in memory).
 * PINGPONG: two buffers; a step reads one and writes the other (pull form).
 * AA: one buffer updated in place, half the memory of PINGPONG. Steps alternate between an
 * even form, in which a site reads its own 27 slots and writes its post-collision values
 * back into the slots of the opposite directions, and an odd form, in which it reads the
 * 27 values its neighbours x - c_i left for it and writes its results into the slots of
 * the neighbours x + c_i. Every site reads and writes the same set of locations, so the
 * update is race-free in place. Both patterns compute identical values (same arithmetic,
 * same Philox counters): only the memory layout between steps differs. AA supports the
 * paper's configuration (omega_g = 1, local rho in Eq. 10) in every storage format. */
typedef enum {
  RFLBM_PATTERN_PINGPONG = 0,
  RFLBM_PATTERN_AA = 1
} rflbm_pattern;

typedef struct {
  int nx, ny, nz;        /* box edges, each >= 1; N = nx*ny*nz < 2^31 */
  double tau;            /* hydrodynamic relaxation time tau_h = 1/omega_h > 1/2 */
  double kT;             /* thermal energy k_B T >= 0 (0: deterministic Reg-LBM) */
  double rho0;           /* reference density > 0 (rest state, storage shift) */
  uint64_t seed;         /* Philox key */
  double omega_g;        /* ghost relaxation rate in (0, 2); the paper uses 1 */
  int model;             /* rflbm_model */
  int storage;           /* rflbm_storage */
  int phi_rho;           /* rflbm_phi_rho */
  uint32_t replica;      /* fourth Philox counter word (independent replicas) */
  void* stream;          /* cudaStream_t for all work, NULL = legacy default stream */
  void* buffers[2];      /* optional caller-owned device buffers of
                            rflbm_buffer_bytes(cfg) bytes each, 256-byte aligned
                            (PINGPONG: both; AA: buffers[0] only, buffers[1] NULL);
                            NULL: the library allocates and frees them */
  int device;            /* CUDA device ordinal, -1 = the current device */
  int kernel;            /* rflbm_kernel */
  int pattern;           /* rflbm_pattern */
  int z0;                /* z-slab: global z of the handle's first row (0 for a whole box) */
  int nz_global;         /* z-slab: z edge of the decomposed box (nx*ny*nz_global < 2^31);
                            0 = the handle holds a whole periodic box (see "z-slabs" below) */
} rflbm_config_t;

typedef struct {
  int64_t step;          /* current step t */
  double mass;           /* sum_s rho(s) (Eq. 3), FP64 accumulation */
  double momentum[3];    /* sum_s rho u(s) (Eq. 4), FP64 accumulation */
  double max_speed;      /* max_s |u(s)| */
  int64_t nonfinite;     /* unstable sites: density or momentum not finite, or density
                            not positive (such sites enter no sum and no max_speed) */
} rflbm_stats_t;

/* Fills cfg with the defaults: 32^3, tau 0.8, kT 0, rho0 1, seed 1, omega_g 1, Reg model,
 * float32 storage, local rho in Eq. 10, replica 0, default stream, library buffers,
 * current device, automatic kernel choice, ping-pong streaming, a whole box (no z-slab). */
void rflbm_config_default(rflbm_config_t* cfg);

/* sizeof(rflbm_config_t) as compiled into the library (for bindings to check their
 * mirror of the struct). */
int64_t rflbm_config_size(void);

/* Bytes of one population buffer for cfg (two are used with PINGPONG, one with AA), or a
 * negative rflbm_status if cfg is invalid. */
int64_t rflbm_buffer_bytes(const rflbm_config_t* cfg);

/* Creates a handle for a periodic box with the paper's defaults (Reg-FLBM, omega_g = 1,
 * Sec. II.B) and the state uninitialised (call an init function before stepping).
 * NULL on error. */
rflbm_t* rflbm_create(int nx, int ny, int nz, double tau, double kT, double rho0,
                      uint64_t seed);

/* Creates a handle from a full configuration. NULL on error. */
rflbm_t* rflbm_create_ex(const rflbm_config_t* cfg);

/* Releases the handle and the device memory the library allocated for it. NULL is a
 * no-op. Waits for the handle's outstanding work. */
void rflbm_destroy(rflbm_t* h);

/* Description of the last error on the calling thread ("" if none). */
const char* rflbm_last_error(void);

/* Fluid at rest: f_i = w_i rho0 (Table I weights; the u = 0 value of Eq. 26); t = 0. */
int rflbm_init_rest(rflbm_t* h);

/* Thermal equilibrium: every mode k of Table II at every site (density and momentum
 * included) an independent normal of variance rho0 kT b_k / cs2 around the rest state,
 * f = w rho0 + w_i sum_k m_k e_ki / b_k (Eq. 11). This is the stationary distribution of
 * the linearised fluctuating model, the per-mode variance the amplitude of Eq. 10
 * maintains (Sec. II.A), so statistics need no burn-in. The draws are Philox4x32-10 calls
 * j = 6..12 at counter (site, 0, j, replica) with the handle's seed (the steps use
 * j = 0..5). kT = 0 gives the rest state. t = 0. Asynchronous on the handle's stream. */
int rflbm_init_thermal(rflbm_t* h);

/* f_i(x, 0) = f_i^(0)(rho(x), u(x)), the equilibrium of Eq. 26; t = 0.
 * rho: N doubles, or NULL for rho0 everywhere; u: 3*N doubles (rows x, y, z), or NULL
 * for rest. Host or device memory per on_device. */
int rflbm_init_field(rflbm_t* h, const double* rho, const double* u, int on_device);

/* Advances n >= 0 steps (Eq. 25, or Eq. 12 for the BGK model, then Eq. 8). Asynchronous
 * on the handle's stream. */
int rflbm_step(rflbm_t* h, int64_t n);

/* Pre-collision moments of the current state, FP64 (Eqs. 3-4; Pi = a^(2) of Sec. III):
 * rho (N), u (3*N, rows x, y, z), pi (6*N, rows xx, yy, zz, xy, xz, yz with
 * Pi_ab = sum_i f_i (c_ia c_ib - cs2 delta_ab)). Any pointer may be NULL to skip that
 * field. Synchronous. */
int rflbm_moments(rflbm_t* h, double* rho, double* u, double* pi, int on_device);

/* Global diagnostics of the current state in FP64 (see rflbm_stats_t). Synchronous.
 * Returns RFLBM_EUNSTABLE (with *out filled) when unstable sites are present. */
int rflbm_stats(rflbm_t* h, rflbm_stats_t* out);

/* Current populations f_i(x, t) as 27*N doubles / floats (layout above). Synchronous.
 * Host memory that is page-locked (cudaHostAlloc, cudaHostRegister) is written by the
 * conversion kernel in place; other host memory goes through a device staging buffer. */
int rflbm_get_populations(rflbm_t* h, double* f, int on_device);
int rflbm_get_populations_f32(rflbm_t* h, float* f, int on_device);

/* Replaces the state by f (27*N doubles / floats) without changing t. Host input is
 * read in place when page-locked, else through the staging buffer; either way the call
 * returns after f has been read. */
int rflbm_set_populations(rflbm_t* h, const double* f, int on_device);
int rflbm_set_populations_f32(rflbm_t* h, const float* f, int on_device);

/* Populations of selected sites: sites (n indices in [0, N), host memory) -> f (27*n
 * doubles in host memory, element [i*n + j] for site sites[j]). Synchronous. */
int rflbm_get_sites(rflbm_t* h, const int64_t* sites, int64_t n, double* f);

/* Checkpoint / resume. rflbm_state_bytes: size of the raw storage image of the state
 * (the shifted populations in the handle's storage format and the library's internal
 * ping-pong layout, 27 planes of rflbm_buffer_bytes / 27 bytes). rflbm_save_state copies
 * that image out, rflbm_load_state replaces the state by an image saved from a handle of
 * the same box and storage format, of either streaming pattern; with rflbm_set_step and
 * the same seed the run continues bit-identically to an uninterrupted one (the noise is
 * keyed by the step). An AA handle after an even number of steps since its state was set
 * writes the image through a one-plane device scratch buffer. */
int64_t rflbm_state_bytes(const rflbm_t* h);
int rflbm_save_state(rflbm_t* h, void* image, int on_device);
int rflbm_load_state(rflbm_t* h, const void* image, int on_device);

/* Step counter: read, and set (checkpoint/resume: with the populations and the seed it
 * reproduces the noise of an uninterrupted run exactly). */
int64_t rflbm_get_step(const rflbm_t* h);
int rflbm_set_step(rflbm_t* h, int64_t step);

/* Changes the stream of all later work (cudaStream_t, NULL = legacy default stream). */
int rflbm_set_stream(rflbm_t* h, void* stream);

/* Waits for all work enqueued on the handle's stream; reports asynchronous errors. */
int rflbm_synchronize(rflbm_t* h);

/* Box edges and number of kernel launches one rflbm_step(h, 1) makes. */
int rflbm_get_dims(const rflbm_t* h, int* nx, int* ny, int* nz);
int rflbm_launches_per_step(const rflbm_t* h);

/* Step kernel the handle runs (an rflbm_kernel value other than AUTO); *width, if not
 * NULL, receives the row-segment width of the TMA kernels (0 for the general kernel). */
int rflbm_step_path(const rflbm_t* h, int* width);

/* Sites one thread of the kernel of the next step (rflbm_step(h, 1)) updates: 2 where the
 * TMA kernels run their two-site form (packed f32x2 arithmetic, one instruction for both
 * sites): Reg-FLBM with 16-bit storage and float32 without noise in either streaming
 * pattern, and the odd AA steps of float32 Reg-FLBM whose rows span several segments; else
 * 1. Both forms compute every site bit for bit alike; negative rflbm_status on an invalid
 * handle. */
int rflbm_step_sites_per_thread(const rflbm_t* h);

/* Equilibrium-statistics diagnostics of the current (pre-collision) state, FP64
 * accumulation, synchronous. They serve the fluctuation-dissipation checks of Sec. III:
 * at equilibrium every mode of Table II fluctuates per site with variance
 * rho0 kT b_k / cs2, and the static structure factors of rho, rho u and Pi are flat.
 *
 * rflbm_mode_sums: sum[k] = sum over sites of m_k - rho0 delta_k0 and sumsq[k] = sum of its
 *   square, for the 27 modes m_k = sum_i e_ki f_i of Table II (Eq. 5); 27 doubles each in
 *   host memory. Per-site values are formed in float32.
 * rflbm_structure_factor: for one field (rflbm_field, per site), F(k) = sum_x phi(x)
 *   exp(-i k.x) by a 3-D FFT (cuFFT), S(k) = |F(k)|^2 / N, summed over the spherical
 *   shells n = round(|k| L / 2 pi), L = max(nx, ny, nz): s_sum[n] = sum of S over the
 *   wave vectors of shell n, count[n] = their number (n < nshell; both host arrays of
 *   nshell doubles; the k = 0 vector is in shell 0). Work buffers (two N-sized FP64 arrays
 *   and the FFT plan) are allocated on first use and kept by the handle.
 * rflbm_shell_count: the number of shells that covers every wave vector of the box. */
typedef enum {
  RFLBM_FIELD_RHO = 0,  /* rho - rho0 */
  RFLBM_FIELD_JX = 1, RFLBM_FIELD_JY = 2, RFLBM_FIELD_JZ = 3,  /* rho u */
  RFLBM_FIELD_PXX = 4, RFLBM_FIELD_PYY = 5, RFLBM_FIELD_PZZ = 6,  /* Pi = a^(2) (Sec. III) */
  RFLBM_FIELD_PXY = 7, RFLBM_FIELD_PXZ = 8, RFLBM_FIELD_PYZ = 9
} rflbm_field;
int rflbm_mode_sums(rflbm_t* h, double* sum, double* sumsq);
int rflbm_structure_factor(rflbm_t* h, int field, int nshell, double* s_sum, double* count);
int rflbm_shell_count(const rflbm_t* h);

/* Test entry points of the noise source (Eq. 9 r_k; the generator is the reading
 * stated above). Host buffers; computed on the current device.
 * rflbm_philox4x32_10: out[4*j + w] = word w of Philox4x32-10(ctr[4*j .. 4*j+3],
 *   key = (k0, k1)) for j < n.
 * rflbm_site_normals: out[24*j + m] = normal n[m] of site sites[j] at (seed, step,
 *   replica), exactly as the step kernel draws it (float32). */
int rflbm_philox4x32_10(const uint32_t* ctr, uint32_t k0, uint32_t k1, uint32_t* out,
                        int64_t n);
int rflbm_site_normals(uint64_t seed, int64_t step, uint32_t replica,
                       const uint32_t* sites, int64_t n, float* out);

/* Batched ensembles: many independent periodic boxes ("replicas") of uneven sizes, seeds,
 * tau and kT, advanced together: each step is one launch over the tiles of every replica,
 * and the n steps of a call replay as one CUDA graph (captured once per n). Each replica
 * runs the Reg-FLBM step of a single box (Eq. 25, omega_g = 1, local rho in Eq. 10) with
 * Philox key = its seed and replica word 0, so it reproduces the run of
 * rflbm_create(nx, ny, nz, tau, kT, rho0, seed) in the same storage format bit for bit.
 * `tile` is the tile size in sites (96, 128, 192, 256 or 512) given to every replica; or -1:
 * each replica takes the first size that its row length divides in the order 128, 96, 192,
 * 256, 512 (float32) or 128, 192, 256, 512, 96 (16-bit storage), and tiles of 128 sites when
 * none does; or 0 (autotuned): the same, except that for each row length that takes row
 * tiles the library times the replicas of that row length alone, a few steps at every size
 * their rows divide, at creation, and keeps the fastest (the state is undefined until the
 * initialisation call that must follow anyway). A replica whose row length nx is at most
 * 256 and a whole number of 16-byte units takes tiles of floor(tile / nx) whole rows moved by
 * TMA copies (run by tile / 2 threads of two sites each in 16-bit storage) when nx divides its
 * tile size or those rows keep at least 85 % of the tile's threads busy (with -1 and 0 such
 * partial tiles are chosen only up to 256 sites, exact divisors first); any other replica
 * takes tiles of `tile` consecutive sites, one thread each. A step is one launch per tile size and
 * kind of tile in use (per group of 64 replicas). A bounded wait for a copy that expires makes
 * the call report RFLBM_ETIMEOUT. The library allocates and owns all device memory. */
typedef struct rflbm_batch rflbm_batch_t;
typedef struct {
  int nx, ny, nz;   /* box edges (N = nx*ny*nz < 2^31) */
  double tau, kT;   /* relaxation time > 1/2, thermal energy >= 0 */
  uint64_t seed;    /* Philox key */
} rflbm_replica_t;
rflbm_batch_t* rflbm_batch_create(const rflbm_replica_t* reps, int n, double rho0, int storage,
                                  int tile);
void rflbm_batch_destroy(rflbm_batch_t* b);
/* The tile size requested at creation (0 or -1: per replica), the resident CTAs per SM of the
 * kernel that updates the most sites, and the tiles per step. */
int rflbm_batch_tuning(const rflbm_batch_t* b, int* tile, int* ctas_per_sm, int64_t* tiles_per_step);
/* Tile size of replica r and its rows per tile (0: tiles of consecutive sites); either
 * pointer may be NULL. */
int rflbm_batch_replica_tiling(const rflbm_batch_t* b, int r, int* tile, int* rows);
/* Kernel launches per step: one per group of 64 replicas, tile size and kind of tile
 * (row tiles, site tiles) in use. */
int rflbm_batch_launches_per_step(const rflbm_batch_t* b);
/* Box edges of replica r (any pointer may be NULL). */
int rflbm_batch_replica_dims(const rflbm_batch_t* b, int r, int* nx, int* ny, int* nz);
/* Every replica at rest, step 0. */
int rflbm_batch_init_rest(rflbm_batch_t* b);
/* n steps of every replica (asynchronous on the default stream). The n steps replay one
 * CUDA graph, captured and instantiated on the host by the first call with this n (the
 * handle keeps the graph of the last n). */
int rflbm_batch_run(rflbm_batch_t* b, int64_t n);
/* Captures and instantiates the graph of an n-step run (n >= 1) without running it, so that
 * the next rflbm_batch_run(b, n) only launches it. Launches nothing. */
int rflbm_batch_prepare(rflbm_batch_t* b, int64_t n);
int rflbm_batch_synchronize(rflbm_batch_t* b);
/* Populations (27*N doubles, public layout) and diagnostics of replica r. Synchronous. */
int rflbm_batch_get_populations(rflbm_batch_t* b, int r, double* f);
int rflbm_batch_stats(rflbm_batch_t* b, int r, rflbm_stats_t* out);

/* z-slabs: one box split along z across several handles (the paper's linear domain
 * decomposition for its multi-GPU runs, Sec. IV), typically one per GPU.
 *
 * A handle created with nz_global > 0 is the z-slab of rows z0 .. z0 + nz - 1 of a periodic
 * box of nx x ny x nz_global sites. Its buffers hold the nz rows between two ghost rows (the
 * row below z0 and the row above z0 + nz - 1), x and y stay periodic inside the handle, and
 * z is periodic across the slabs. The noise of a site is keyed by its global index
 * x + nx (y + ny z) (rflbm.h conventions), so slabs that exchange their faces after every
 * step reproduce the run of the undecomposed box bit for bit, in both streaming patterns
 * and every storage format. Sites, fields and populations of the public layout are the
 * slab's own nx*ny*nz sites. rflbm_step takes one step per call on a slab: it updates the
 * two boundary rows first and then the interior rows, so that the faces can move while the
 * interior updates. Until the exchange of that step is complete, the slab accepts no other
 * call that reads or advances its state (RFLBM_ESTATE). The structure factor needs the
 * whole box and is not available on a slab; state images of AA slabs are not supported.
 *
 * A face is 9 rows of nx*ny values (the populations with c_z = +1 going up, or c_z = -1
 * going down), given as three runs of three planes: run r starts at run[r]; plane p of the
 * run (p = 0, 1, 2) starts plane_pitch * p bytes further; each plane row is row_bytes
 * contiguous bytes of device memory of the handle's device. After each step, the bytes of
 * send_up must reach the upper neighbour's recv_below and those of send_down the lower
 * neighbour's recv_above, run by run and plane by plane (the neighbours of the top and the
 * bottom slab wrap around periodically). Which rows these are depends on the pattern and
 * the step's parity: query them after every step. */
typedef struct {
  void* run[3];          /* first byte of each run of three plane rows */
  int64_t plane_pitch;   /* bytes from one plane row of a run to the next */
  int64_t row_bytes;     /* contiguous bytes of one plane row (nx*ny values) */
} rflbm_face_t;

/* The four faces of the exchange that the slab's last step requires (any pointer may be
 * NULL). RFLBM_ESTATE if no exchange is pending, RFLBM_EINVAL for a handle that is not a
 * slab. */
int rflbm_slab_faces(rflbm_t* h, rflbm_face_t* send_up, rflbm_face_t* send_down,
                     rflbm_face_t* recv_below, rflbm_face_t* recv_above);
/* Makes `stream` (a cudaStream_t of the handle's device) wait until the boundary rows of
 * the slab's last step are written: work enqueued on it afterwards may read the send faces
 * and write the receive faces. */
int rflbm_slab_faces_ready(rflbm_t* h, void* stream);
/* Declares the exchange complete once the work enqueued on `stream` so far has run: the
 * slab's next work waits for it, and its state may be read and stepped again. */
int rflbm_slab_exchange_done(rflbm_t* h, void* stream);
/* The whole exchange for n slabs of one box on one device, given in z order (slab k + 1 is
 * above slab k, the last below the first): device-to-device copies (one 3-D copy per face
 * while its plane pitch is within the device's maximum copy pitch, else one per plane row)
 * on a stream of the library that waits for every slab's boundary rows and overlaps their
 * interior rows; then every slab's next step waits for the copies. n = 1 makes one slab
 * periodic in z. */
int rflbm_slab_exchange(rflbm_t* const* slabs, int n);

/* Global diagnostics of caller-owned populations that allocate nothing.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory at the moment they need these numbers, typically because their
 * framework has already reserved the device memory for its own pool (a cudaMalloc would
 * fail, or would synchronise the device inside a pipeline that must not stall), or
 * because they run as a hook between the steps of another solver. It computes what
 * rflbm_stats computes (FP64 sums of density and momentum, maximum speed, unstable
 * sites; step is set to 0) for populations in the public layout: f holds 27 planes of
 * n_sites float32 values in device memory of the current device (element [i*n_sites + s]),
 * owned by the caller. `stream` is a cudaStream_t or NULL; the call waits for it and fills
 * *out (host memory).
 *
 * Scratch: a fixed area in the library's static device memory (about 512 KB, held by
 * every GPU that loads the library until the process exits); no cudaMalloc, cudaFree or
 * other allocating routine is called. Capacity: n_sites <= RFLBM_STATS_NOALLOC_MAX_SITES
 * (8192 partial sums of 16384 sites); larger inputs are rejected with RFLBM_EINVAL. Every
 * call looks up the area's device address on the current device (cudaGetSymbolAddress,
 * which allocates nothing), so a call stays valid after a cudaDeviceReset. All calls share the
 * area: calls that overlap on the GPU (two streams or two host threads at once) race and
 * must be serialised by the caller. Returns RFLBM_OK, RFLBM_EUNSTABLE (unstable sites;
 * *out filled), RFLBM_EINVAL or RFLBM_ECUDA (message in rflbm_last_error). */
#define RFLBM_STATS_NOALLOC_MAX_SITES 134217728LL
int rflbm_stats_f32_noalloc(const float* f, int64_t n_sites, void* stream, rflbm_stats_t* out);

#ifdef __cplusplus
}
#endif

#endif /* RFLBM_H */
