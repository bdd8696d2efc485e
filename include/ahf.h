/*
 * libahfgpu - C ABI of the per-halo unbinding stage of AHF
 * (Knollmann & Knebe 2009, "AHF: Amiga's Halo Finder"), for one GB300 GPU.
 *
 * What the library computes, per candidate halo (Sect. 2.1 and Appendix A):
 *   1. gather: the candidates of the halo inside its gather sphere
 *      |x - c| <= R, recentred in FP64 (minimum image in a periodic box);
 *   2. sort the members once by radius (ties by candidate position);
 *   3. iterate: potential phi_i = -G [M(<r_i)/r_i + sum_{j>=i} m_j/r_j]
 *      (Appendix A, Eqs. A1-A4 with phi_0 from Eq. A9, the halo truncated at
 *      its outermost member), escape test |v - v_bulk + H d|^2 > 2|phi|
 *      (v_esc = sqrt(2|phi|), Appendix A), simultaneous removal of every
 *      unbound particle, until an iteration removes nothing;
 *   4. virial radius and mass of the final set: the first outward crossing
 *      of the mean enclosed density through delta_rho (Sect. 2.1, Eqs. 1-2);
 *   5. optionally a log-radial profile of the bound set (Sect. 2.1, the
 *      radially binned halo output).
 *
 * Conventions shared by every entry point
 *   - Every call returns an int: AHF_OK (0), AHF_PENDING (1, polling only),
 *     or a negative AHF_ERR_* code.  No C++ exception crosses the ABI and no
 *     call aborts the process.  ahf_last_error() returns a thread-local,
 *     human-readable message for the last failing call on that thread.
 *   - Buffers are owned by the caller unless stated otherwise.  "device"
 *     means memory of the context's GPU (cudaMalloc, torch.cuda, managed);
 *     "host" means ordinary or pinned CPU memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls enqueue their work on it and return; results are
 *     valid once the stream has reached that point.  A call whose batch
 *     holds haloes above the on-chip size class synchronises `stream`
 *     between iterations of that class (convergence is decided on the host).
 *   - Candidate slots.  Halo h owns the slots [offset, offset + count).
 *     Without a member list, slot s is particle s; with a member list,
 *     slot s is particle member_idx[s].  Haloes must not share slots.
 *     Per-slot outputs (bound_idx, phi, removed_iter) use the same slots:
 *     halo h writes its k-th bound particle at slot offset + k.
 */
#ifndef AHF_H
#define AHF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ------------------------------------------------------ */
#define AHF_OK            0
#define AHF_PENDING       1
#define AHF_ERR_INVALID   (-1)   /* bad argument, size or layout           */
#define AHF_ERR_NOMEM     (-2)   /* device allocation failed / above a cap */
#define AHF_ERR_TIMEOUT   (-3)   /* a bounded device wait gave up          */
#define AHF_ERR_CUDA      (-4)   /* a CUDA runtime call failed             */
#define AHF_ERR_FULL      (-5)   /* serving queue full                     */
#define AHF_ERR_NOT_FOUND (-6)   /* unknown request id                     */

/* ---- per-halo status bits (ahf_result.status) --------------------------- */
#define AHF_HALO_OK               0
#define AHF_HALO_NOT_CONVERGED    1  /* max_iter reached while still removing */
#define AHF_HALO_EMPTY            2  /* no member left                        */
#define AHF_HALO_RVIR_BEYOND_EDGE 4  /* mean density above delta_rho at the outermost member */
#define AHF_HALO_RVIR_NONE        8  /* mean density never reaches delta_rho  */
#define AHF_HALO_RISE_EDGE       16  /* extent at the rise of the density
                                        profile (AHF_VAR_RISE_EDGE)           */

/* ---- coordinate encodings (ahf_particles.coord_type) -------------------- */
#define AHF_COORD_F64     0  /* double x,y,z,vx,vy,vz,m; any frame           */
#define AHF_COORD_F32_REL 1  /* float; positions already near the centre    */
#define AHF_COORD_F32_BOX 2  /* float box coordinates (e.g. [0, box))       */

/* ---- precision modes (ahf_params.precision) ----------------------------- */
/* MIXED: FP64 recentring, FP32 per-particle arithmetic, and every sum that
 * needs more than FP32 (M(<r), sum m/r, sum m v, sum m) accumulated exactly
 * in 64-bit fixed point, which is at least as accurate as FP64 here and
 * independent of summation order.  FP64: the same with FP64 per-particle
 * arithmetic (phi and the escape test in double). */
#define AHF_PREC_MIXED 0
#define AHF_PREC_FP64  1

typedef struct ahf_params {
  double G;          /* gravitational constant in the caller's units            */
  double H;          /* Hubble constant: the escape test uses u = v - v_bulk + H d */
  double delta_rho;  /* Delta * rho_b of Eq. 1 (mass / length^3)                */
  double r_soft;     /* radius floor: every r is replaced by max(r, r_soft); with
                        0, pair terms with max(r_i, r_j) = 0 are dropped        */
  double box;        /* periodic box size; 0 = not periodic                     */
  double band;       /* relative half-width of the reported decision band,
                        |(|u|^2 - 2|phi|) / 2|phi|| < band (default 1e-5)      */
  int32_t max_iter;  /* iteration cap (>= 1)                                    */
  int32_t precision; /* AHF_PREC_MIXED or AHF_PREC_FP64                         */
  int32_t variant;   /* AHF_VAR_* bits (0: the method as described above)       */
  int32_t reserved;  /* must be 0                                               */
} ahf_params;

/* ---- method variants (ahf_params.variant) ---------------------------------
 * AHF_VAR_VBULK_INITIAL: the escape test uses the bulk velocity of the
 *   initial member set in every iteration instead of the current set's.
 * AHF_VAR_RETRUNCATE: after the unbinding converges, each halo with an r_vir
 *   is cut to its bound particles within r_vir and unbound again (Appendix A
 *   truncates the potential at r_vir).  Records, bound lists, phi and profile
 *   rows describe the second pass; removed_iter keeps the first pass's
 *   removals (candidates outside r_vir or removed by the second pass appear
 *   only as missing from the bound list).  The call then reads the first
 *   pass's records back to the host (it synchronises `stream` once).
 *   ahf_unbind_batch, ahf_unbind_profile_batch and ahf_unbind_batch_host
 *   only.
 * AHF_VAR_RISE_EDGE: a halo whose mean overdensity never drops below
 *   delta_rho inside its bound set (AHF_HALO_RVIR_BEYOND_EDGE) ends at the rise
 *   of its density profile (Sect. 2.1, the truncation of subhaloes): the bound
 *   set, sorted by radius, is cut into 16 shells of equal particle count; among
 *   the outer 8 shells the first of least density (shell mass over the volume
 *   between the radii of the last particles of the shell and of the one
 *   before) is the edge when a denser shell lies beyond it.  k_vir is then the
 *   shell's last particle, r_vir its radius, m_vir the mass up to it, and the
 *   status gains AHF_HALO_RISE_EDGE.  Bound sets of fewer than 64 particles
 *   are left as they are.  The profile rows use that r_vir. */
#define AHF_VAR_VBULK_INITIAL 1
#define AHF_VAR_RETRUNCATE    2
#define AHF_VAR_RISE_EDGE     4

typedef struct ahf_particles {
  /* Structure-of-arrays particle store, n entries each.  Element type is
     double for AHF_COORD_F64 and float otherwise.  m may be NULL: every
     particle then has mass m0. */
  const void *x, *y, *z, *vx, *vy, *vz, *m;
  double m0;
  int64_t n;
  int32_t coord_type;
  int32_t reserved;  /* must be 0 */
  /* Specific thermal energy of gas (SPH) particles, velocity^2 units, 0 for
     collisionless ones; NULL = none.  With it the escape test is
     |u|^2 + 2 u_th > 2|phi| (Sect. 2.1: the thermal energy of gas particles
     counts in the unbinding), and every halo takes the multi-CTA class. */
  const void *u_th;
} ahf_particles;

typedef struct ahf_halo {
  double cx, cy, cz; /* centre, same frame as the particle coordinates (FP64) */
  double radius;     /* gather-sphere radius R; members satisfy |x - c| <= R  */
  int64_t offset;    /* first candidate slot                                  */
  int64_t count;     /* number of candidate slots (>= 0)                      */
} ahf_halo;

typedef struct ahf_result {
  int64_t n_bound;   /* members left after unbinding                          */
  int64_t n_member;  /* candidates inside the gather sphere                   */
  int64_t part_iter; /* sum over iterations of the members tested             */
  int64_t n_band;    /* sum over iterations of tests inside the band          */
  int64_t k_vir;     /* index in the sorted bound list of the last particle
                        inside r_vir, -1 if none                              */
  int32_t n_iter;    /* iterations run, the last one removing nothing unless
                        AHF_HALO_NOT_CONVERGED                                */
  int32_t status;    /* AHF_HALO_* bits                                       */
  double m_vir;      /* M_vir = M(<= r_vir) (Eq. 2)                           */
  double r_vir;      /* r_vir with M_vir / (4/3 pi r_vir^3) = delta_rho (Eq. 1) */
  double vbulk[3];   /* mass-weighted mean velocity of the bound set          */
} ahf_result;        /* 88 bytes */

typedef struct ahf_ctx ahf_ctx;

/* Library version (major * 10000 + minor * 100 + patch). */
int ahf_version(void);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *ahf_last_error(void);

/* Create a context on CUDA device `device`.  The context owns its device
 * workspace (grown on demand, released by ahf_destroy) and its streams.
 * Tuning: when the environment variable AHF_TUNING names a file written by
 * the autotuner (paper_0904_3662_gb300/autotune.py: lines "device <name>",
 * "build <id>", "option <number> <value>"), its options are applied if its
 * device name and build id are this device's and ahf_build_id()'s, and
 * ignored otherwise; ahf_set_option overrides them afterwards.
 * Errors: AHF_ERR_INVALID (ctx NULL, bad device, a tuning file that does
 * not parse), AHF_ERR_CUDA. */
int ahf_create(ahf_ctx **ctx, int device);

/* Identifier of this build of the library (a hash of its sources), which
 * tuning files are keyed by. */
const char *ahf_build_id(void);

/* Release the context and its workspace; waits for its work to finish.
 * NULL is accepted. */
int ahf_destroy(ahf_ctx *ctx);

/* Iterative unbinding of a batch of haloes (Sect. 2.1 and Appendix A).
 *   p            particle store (device pointers), see ahf_particles
 *   halos        host array of n_halos descriptors
 *   member_idx   device int64 slot -> particle index map, or NULL (slot = particle)
 *   prm          host parameters
 *   out          device array of n_halos ahf_result records
 *   bound_idx    device int64 per slot: halo h writes the particle indices of
 *                its bound set, sorted by (radius, slot), at offset..offset+n_bound-1
 *   phi          device per slot, nullable: phi of each bound particle, aligned
 *                with bound_idx (float for MIXED, double for FP64)
 *   removed_iter device int32 per slot, nullable: -1 outside the gather sphere,
 *                0 bound, t > 0 removed in iteration t
 * Slots of a halo beyond offset + n_bound are left unspecified in bound_idx
 * and phi.  Errors: AHF_ERR_INVALID (NULL pointers, negative sizes, n_halos
 * of 2^27 or more, slots out of range or shared, bad coord_type/precision/
 * max_iter), AHF_ERR_NOMEM, AHF_ERR_CUDA (AHF_ERR_TIMEOUT through ahf_sync).
 * Outputs are undefined after an error. */
int ahf_unbind_batch(ahf_ctx *ctx, const ahf_particles *p, const ahf_halo *halos,
                     int64_t n_halos, const int64_t *member_idx, const ahf_params *prm,
                     ahf_result *out, int64_t *bound_idx, void *phi,
                     int32_t *removed_iter, void *stream);

/* The same computation with every pointer in HOST memory (pageable or
 * pinned): the call stages the inputs on the device, runs ahf_unbind_batch
 * and, when n_bins > 0, ahf_profile_batch into `prof` (host double
 * [n_halos][n_bins][4], may be NULL when n_bins is 0), copies the outputs
 * back and returns when they are in place (it synchronises `stream`).
 * Same arguments, layouts and errors as the two device entry points. */
int ahf_unbind_batch_host(ahf_ctx *ctx, const ahf_particles *p, const ahf_halo *halos,
                          int64_t n_halos, const int64_t *member_idx, const ahf_params *prm,
                          ahf_result *out, int64_t *bound_idx, void *phi,
                          int32_t *removed_iter, int32_t n_bins, double r_min_frac,
                          double *prof, void *stream);

/* Plain form of the same stage: one halo at a time, separate kernel launches
 * for gather, sort and each iteration's scan / test / compaction, and a host
 * synchronisation on every iteration's change flag.  Same arguments, results
 * and errors as ahf_unbind_batch; it exists as the one-halo-per-launch
 * baseline the batched form is measured against. */
int ahf_unbind_plain(ahf_ctx *ctx, const ahf_particles *p, const ahf_halo *halos,
                     int64_t n_halos, const int64_t *member_idx, const ahf_params *prm,
                     ahf_result *out, int64_t *bound_idx, void *phi,
                     int32_t *removed_iter, void *stream);

/* Log-radial profile of bound sets (Sect. 2.1: the radially binned output).
 *   p, halos, n_halos, member_idx, prm   as passed to ahf_unbind_batch
 *   res, bound_idx                       its outputs (device)
 *   n_bins (1..4096), r_min_frac (0 < f < 1)
 *   prof  device double [n_halos][n_bins][4]
 * Bin b of halo h covers (e_b, e_{b+1}] with e_b = r_out f^(1 - b/n_bins),
 * r_out = r_vir, or the outermost bound radius when r_vir is 0.  Columns:
 * count, mass within e_{b+1}, mass of the bin / shell volume, circular
 * velocity sqrt(G M(<= e_{b+1}) / e_{b+1}).  Empty haloes give zero rows.
 * Errors: AHF_ERR_INVALID, AHF_ERR_NOMEM, AHF_ERR_CUDA. */
int ahf_profile_batch(ahf_ctx *ctx, const ahf_particles *p, const ahf_halo *halos,
                      int64_t n_halos, const int64_t *member_idx, const ahf_params *prm,
                      const ahf_result *res, const int64_t *bound_idx, int32_t n_bins,
                      double r_min_frac, double *prof, void *stream);

/* Wait for the context's enqueued work and report problems the device
 * found while running it: AHF_ERR_INVALID for an out-of-range member index
 * or a halo routed to a class it did not fit, AHF_ERR_TIMEOUT when a warp of
 * the multi-CTA passes gave up waiting for its tensor copy into shared
 * memory (AHF_OPT_WAIT_LIMIT; the results of that call are then undefined).
 * The device error word is cleared by the call.  No kernel waits for
 * another CTA. */
int ahf_sync(ahf_ctx *ctx);

/* ahf_unbind_batch and ahf_profile_batch in one call: the same arguments
 * and outputs as the two (prof: device double [n_halos][n_bins][4]).  Haloes
 * small enough for one warp or one CTA get their profile rows from the
 * unbinding kernel itself (the bound set is still on chip); the others get
 * them from the profile kernels.  Rows agree with ahf_profile_batch: counts
 * exactly, masses to rounding (exact fixed-point sums here, FP64 sums there).
 * Errors: those of the two calls. */
int ahf_unbind_profile_batch(ahf_ctx *ctx, const ahf_particles *p, const ahf_halo *halos,
                             int64_t n_halos, const int64_t *member_idx, const ahf_params *prm,
                             ahf_result *out, int64_t *bound_idx, void *phi,
                             int32_t *removed_iter, int32_t n_bins, double r_min_frac,
                             double *prof, void *stream);

/* Tuning and diagnostics knobs (values persist in the context).
 *   AHF_OPT_ONCHIP_MAX   largest candidate count handled in shared memory (by one
 *                        CTA or one thread-block cluster); larger haloes take the
 *                        multi-CTA class (default and maximum 131072)
 *   AHF_OPT_WAIT_LIMIT   polls a warp of the multi-CTA passes makes of the
 *                        barrier of its shared-memory tensor copy before it
 *                        gives up and reports AHF_ERR_TIMEOUT (through
 *                        ahf_sync); 0 = give up at once.  Default 2^22.
 *   AHF_OPT_TIMING       1 = record CUDA events around every phase of the
 *                        following calls (read with ahf_get_stats), 0 = off
 *   AHF_OPT_GRAPHS       1 = a batch whose haloes all take the on-chip classes
 *                        runs its launches as a CUDA graph, captured once and
 *                        replayed while the launch parameters (buffers, class
 *                        sizes, grid shapes) repeat; 0 (default) = plain
 *                        launches.  Ignored while AHF_OPT_TIMING is on.
 *   AHF_OPT_TRACE        1 = the on-chip kernels of the following calls record
 *                        per-halo timestamps (read with ahf_get_trace), 0 = off
 *   AHF_OPT_SERIAL       1 = the on-chip size classes run one after another on
 *                        the caller's stream, so that each phase's events time
 *                        its kernel alone (as a profiler's launch list does);
 *                        0 (default) = concurrently on side streams.  Results
 *                        are the same bits either way.
 *   AHF_OPT_PROMOTE      1 (default) = a batch that would leave SMs idle runs its
 *                        haloes in larger size classes (up to two classes up,
 *                        more threads per halo, lower latency) as long as the
 *                        whole batch still runs at once; 0 = every halo in the
 *                        smallest class that holds it.  Results are the same
 *                        bits either way.
 *   AHF_OPT_PASS_CHUNK   multi-CTA passes enqueued between reads of the count
 *                        of still-active haloes (1..64, default 8; a pass with
 *                        nothing left to do returns at once)
 *   AHF_OPT_WORKSPACE_CAP largest device workspace (bytes) the context may
 *                        hold; a call that needs more fails with
 *                        AHF_ERR_NOMEM before enqueuing anything (0, the
 *                        default: no cap)
 *   AHF_OPT_CLASS_CUT+v  largest candidate count routed to on-chip variant v
 *                        (v = 0..7, the phases 0-7 of ahf_stats; 0..its
 *                        capacity, default the capacity; 0 = none): haloes go
 *                        to the first variant whose cut holds them, else to
 *                        the multi-CTA class.  Every routing gives the same
 *                        results bit for bit (exact sums); only the time
 *                        changes.  These are the autotuner's knobs.
 *   AHF_OPT_HOST_DIRECT  ahf_unbind_batch_host only, for buffers that are
 *                        page-locked (cudaHostAlloc, cudaHostRegister; pageable
 *                        buffers are always staged): 0 = stage every input in
 *                        device memory before the kernels and copy every
 *                        output back after them; 1 = the kernels read
 *                        the inputs and write the outputs in place through
 *                        their mapped device addresses, with no staging of
 *                        the inputs (for inputs too large to stage; slower:
 *                        the kernels' scattered output writes cross the host
 *                        link one by one); 2 = the kernels read the inputs in
 *                        place (each candidate once, over the host link, while
 *                        other haloes compute), and each size class copies its
 *                        haloes' bound lists, phi and removal iterations to
 *                        the caller's buffers as soon as its kernel is done,
 *                        while the others still run (the records and profile
 *                        rows follow at the end; outputs that are not
 *                        page-locked, and the two-pass truncation variant,
 *                        are copied back at the end as in 0).  Default 2.
 * Errors: AHF_ERR_INVALID (unknown option or value). */
#define AHF_OPT_ONCHIP_MAX 1
#define AHF_OPT_WAIT_LIMIT 2
#define AHF_OPT_TIMING     3
#define AHF_OPT_HOST_DIRECT 4
#define AHF_OPT_GRAPHS     5
#define AHF_OPT_TRACE      6
#define AHF_OPT_SERIAL     7
#define AHF_OPT_PROMOTE    8
#define AHF_OPT_PASS_CHUNK 9
#define AHF_OPT_WORKSPACE_CAP 10
#define AHF_OPT_CLASS_CUT  16   /* 16 + v, v = 0..7 */

/* Per-call statistics of the most recent unbinding or profile call.
 * Phases: 0 the warp variant (one warp per halo, 512 slots), 1-3 the
 * single-CTA shared-memory variants (1k / 4k / 8k slots), 4-7 the cluster
 * variants (2 / 4 / 8 / 16 CTAs, 16k / 32k / 64k / 128k slots), 8 the
 * multi-CTA class's gather + sort + fill, 9 its iterations, 10 its final
 * pass, 11 the profile.  phase_ms is device time between events recorded on the stream
 * the phase ran on (valid only with AHF_OPT_TIMING on; -1 otherwise);
 * phase_halos / phase_candidates count the haloes and candidate slots each
 * phase covered. */
#define AHF_N_PHASES 12
typedef struct ahf_stats {
  int64_t launches;                    /* kernels launched by the call        */
  int64_t host_syncs;                  /* host synchronisations in the call   */
  int64_t grid_iterations;             /* multi-CTA iterations launched       */
  int64_t phase_halos[AHF_N_PHASES];
  int64_t phase_candidates[AHF_N_PHASES];
  double phase_ms[AHF_N_PHASES];
  int64_t graph_launches;              /* CUDA graph launches by the call     */
  int64_t graph_captures;              /* graphs captured (new launch key)    */
} ahf_stats;

/* Per-halo trace of the last unbinding call made with AHF_OPT_TRACE on: for
 * every halo (caller's order) AHF_TRACE_FIELDS int64 values,
 *   0 start, 1 gathered, 2 sorted, 3 filled, 4 iterated, 5 done
 *     (device global timer, ns, read by the halo's first thread),
 *   6 the SM that ran the halo's first thread,
 *   7 variant (the phase index of ahf_stats) + 256 * iterations.
 * Haloes of the multi-CTA class have all fields 0.  Waits for the call's
 * device work.  Errors: AHF_ERR_INVALID (NULL, n_halos not the last call's,
 * tracing was off), AHF_ERR_CUDA. */
#define AHF_TRACE_FIELDS 8
int ahf_get_trace(ahf_ctx *ctx, int64_t *host, int64_t n_halos);

/* Copy the statistics of the context's last call (waits for its device work
 * when timing is on).  Errors: AHF_ERR_INVALID (NULL), AHF_ERR_CUDA. */
int ahf_get_stats(ahf_ctx *ctx, ahf_stats *out);
int ahf_set_option(ahf_ctx *ctx, int option, int64_t value);
int ahf_get_option(ahf_ctx *ctx, int option, int64_t *value);

/* Allocation-free unbinding for callers that cannot let a library allocate.
 *
 * Which callers: applications that have given all device memory to their own
 * allocator (a framework's caching allocator, a serving engine's fixed pool)
 * and loops that must never block in cudaMalloc / cudaFree, which
 * synchronise the whole device.  This entry point needs no context and
 * allocates nothing, on the device or on the host.  It computes exactly what
 * ahf_unbind_batch computes (same arguments, layouts and results) for
 * batches whose haloes all fit the on-chip class.  The paper has no
 * counterpart: it is an interface choice of this library.
 *
 * Limits: n_halos <= AHF_STATIC_MAX_HALOS and every halo's count <=
 * AHF_STATIC_MAX_COUNT; larger requests return AHF_ERR_INVALID before any
 * work is enqueued.  Only AHF_PREC_MIXED, no gas (u_th), and of the
 * variants only AHF_VAR_VBULK_INITIAL and AHF_VAR_RISE_EDGE.
 *
 * Scratch: the halo descriptors and work counters live in one fixed array
 * in device memory (about 3.8 MiB) that every GPU loading the library holds
 * until the process exits.  All calls on a device share it and it keeps the
 * last call's contents; each call clears the counters it uses.  Calls whose
 * device work overlaps (different streams with no ordering between them)
 * race on the array and give undefined results: serialise them.
 *
 * Set-up: the first call on a device (the current device, cudaGetDevice)
 * looks up the array's device address with cudaGetSymbolAddress; make that
 * first call before any stream capture.  The descriptors are staged through
 * a host array that the next call overwrites, so the call returns
 * AHF_ERR_INVALID, having enqueued nothing, while `stream` is being
 * captured.  The call runs on `stream` and returns without waiting.
 *
 * error_out: device int32, nullable.  When given, a last kernel on `stream`
 * writes AHF_OK there, or AHF_ERR_INVALID when a member index was out of
 * range (that candidate was treated as outside the gather sphere).
 * Errors: AHF_ERR_INVALID, AHF_ERR_CUDA; ahf_last_error() has the message. */
#define AHF_STATIC_MAX_HALOS 32768
#define AHF_STATIC_MAX_COUNT 8192
int ahf_unbind_batch_static(const ahf_particles *p, const ahf_halo *halos, int64_t n_halos,
                            const int64_t *member_idx, const ahf_params *prm, ahf_result *out,
                            int64_t *bound_idx, void *phi, int32_t *removed_iter, int32_t *error_out,
                            void *stream);

/* ---- hosts and subhaloes ------------------------------------------------------ */

/* Unbinding in dependency order (Sect. 2.1): parent[h] is the host of halo h
 * (-1: a field halo); haloes are unbound deepest level first, and a halo's
 * candidates lose the particles that any of its descendants bound (the
 * paper's option of not including subhaloes in their hosts; particles a
 * subhalo does not bind remain its host's candidates).  After each level a
 * particle's owner is the halo of that level that bound it (the highest
 * index if several did); a candidate is dropped from halo h when its owner
 * descends from h.  Haloes share particles through member lists (their slots
 * stay distinct).  Same buffers and results as ahf_unbind_batch, dropped
 * candidates reported like those outside the sphere (removed_iter -1).  The
 * call reads each level's kept-candidate counts back to the host (one
 * stream synchronisation per level).  Not with AHF_VAR_RETRUNCATE.
 * Errors: those of ahf_unbind_batch; AHF_ERR_INVALID for parent indices out
 * of range or forming a cycle. */
int ahf_unbind_hierarchy(ahf_ctx *ctx, const ahf_particles *p, const ahf_halo *halos, int64_t n_halos,
                         const int64_t *parent, const int64_t *member_idx, const ahf_params *prm,
                         ahf_result *out, int64_t *bound_idx, void *phi, int32_t *removed_iter,
                         void *stream);

/* ---- integral properties and catalogue matching --------------------------- */

/* Integral properties of the bound sets an unbinding call produced (Sect.
 * 3.1: the spin parameter lambda = J sqrt|E| / (G M^(5/2)); the rotation
 * curve's peak).  Over the material within r_vir -- the first k_vir + 1
 * particles of a halo's bound list, or the whole bound list when the halo has
 * no r_vir -- with d the offset from the centre (FP64, minimum image),
 * v_bar = sum m v / M, u = v - v_bar + H d (the unbinding's frame):
 *   M = sum m, J = sum m d x u, K = sum m |u|^2 / 2, U = sum m phi / 2
 *   (phi: the unbinding's output), E = K + U,
 *   v_c(r_i) = sqrt(G M(<= r_i) / r_i) along the radial order, v_max its
 *   maximum and r_max the first radius reaching it.
 *   p, halos, n_halos, member_idx, prm   as passed to ahf_unbind_batch
 *   res, bound_idx, phi                  its outputs (device; phi float in
 *                                        the mixed mode, double in FP64)
 *   props   device double [n_halos][AHF_PROP_FIELDS]:
 *           0 n used, 1 M, 2-4 J, 5 K, 6 U, 7 E, 8 lambda, 9 v_max, 10 r_max,
 *           11 1 if the set was cut at r_vir, else 0
 * Sums are FP64 in a fixed order (repeatable bit for bit).  Empty haloes give
 * zero rows.  Errors: AHF_ERR_INVALID, AHF_ERR_NOMEM, AHF_ERR_CUDA. */
#define AHF_PROP_FIELDS 12
int ahf_halo_properties(ahf_ctx *ctx, const ahf_particles *p, const ahf_halo *halos, int64_t n_halos,
                        const int64_t *member_idx, const ahf_params *prm, const ahf_result *res,
                        const int64_t *bound_idx, const void *phi, double *props, void *stream);

/* Cross-identification of two catalogues (Sect. 3.2): for every halo a of
 * the first, the halo b of the second maximising xi = N_shared^2 / (N_a N_b),
 * N_shared the particle ids the two have in common (ties: the lower b).
 * Catalogue X holds halo k's ids at ids_x[off_x[k] .. off_x[k] + cnt_x[k]);
 * ids lie in [0, n_ids), are distinct within a halo, and each id belongs to
 * at most one halo of the second catalogue (pass exclusive membership lists).
 * All arrays are device memory.  Outputs over the first catalogue (device):
 * best (-1: no shared id), shared, xi (0 when best is -1).  The context's
 * workspace holds one int per id.  Problems the device finds (an id out of
 * range, an id in two haloes of the second catalogue, a halo meeting more
 * than 2048 haloes, whose best is then -2) are reported by ahf_sync as
 * AHF_ERR_INVALID.  Errors: AHF_ERR_INVALID, AHF_ERR_NOMEM, AHF_ERR_CUDA. */
int ahf_match_catalogs(ahf_ctx *ctx, int64_t n_ids, const int64_t *ids_a, const int64_t *off_a,
                       const int64_t *cnt_a, int64_t n_a, const int64_t *ids_b, const int64_t *off_b,
                       const int64_t *cnt_b, int64_t n_b, int64_t *best, int64_t *shared, double *xi,
                       void *stream);

/* ---- serving: continuous batching of one-halo requests --------------------
 *
 * For callers that produce candidate haloes over time rather than as one
 * snapshot (the paper analyses a snapshot in one pass and has no such
 * layer).  A request is one halo with its candidates; a worker thread packs
 * the queued requests into batches and runs them through ahf_unbind_batch,
 * forming and copying the next batch while the previous one computes.  A
 * request's result is identical to unbinding that halo alone: every halo is
 * computed independently and order-independently.
 *
 * Memory: a request holds candidate slots from submission until its batch
 * has completed, in two rings.  The device ring is sized from hbm_cap_bytes
 * (device bytes for the particle state and bound lists of every request in
 * flight, the result records and the context's workspace): a request that
 * does not fit in the device memory left is refused with AHF_ERR_FULL.  A
 * pinned host ring of at most 2^23 slots stages the candidates and takes the
 * bound lists back; it refuses the same way when full.  A request holds
 * max(count, 1) slots of each; slots return in submission order. */
typedef struct ahf_serve ahf_serve;

/* Create a serving instance on `device` with parameters `prm` (copied).
 * Every request uses coordinate encoding `coord_type`; m0 > 0 means every
 * particle has mass m0 and requests carry no masses, m0 == 0 means every
 * request carries per-particle masses.  Starts the worker thread.
 * Errors: AHF_ERR_INVALID (NULL, bad params or coord_type, a cap too small
 * for a request of AHF_SERVE_MAX_COUNT candidates), AHF_ERR_NOMEM,
 * AHF_ERR_CUDA. */
#define AHF_SERVE_MAX_COUNT 131072
int ahf_serve_create(ahf_serve **s, int device, size_t hbm_cap_bytes, const ahf_params *prm,
                     int32_t coord_type, double m0);

/* Submit one halo.  p: HOST particle arrays (coord_type and masses as the
 * instance takes them); halo: centre, gather radius, and the candidates
 * [offset, offset + count) of p (count <= AHF_SERVE_MAX_COUNT).  The
 * candidates are copied before the call returns, so the caller may reuse p.
 * On success *req_id identifies the request.  Never blocks on the GPU.
 * Requests carry no gas thermal energies (u_th must be NULL).
 * Errors: AHF_ERR_INVALID, AHF_ERR_NOMEM, AHF_ERR_FULL (no room in the ring
 * now: poll completed requests and retry). */
int ahf_serve_submit(ahf_serve *s, const ahf_particles *p, const ahf_halo *halo, uint64_t *req_id);

/* Non-blocking: AHF_PENDING while the request runs; AHF_OK once it has
 * completed, after writing its record to *out_host (nullable) and its bound
 * list, sorted by radius and given as indices into the submitted p, to
 * bound_idx_host[0 .. n_bound) (nullable; cap entries available).  A
 * completed request is forgotten after AHF_OK (a second poll returns
 * AHF_ERR_NOT_FOUND).  Errors: AHF_ERR_NOT_FOUND, AHF_ERR_INVALID (cap below
 * n_bound: *out_host is written, the request is kept, poll again with a
 * larger buffer), or the error that failed the request's batch (the request
 * is then forgotten). */
int ahf_serve_poll(ahf_serve *s, uint64_t req_id, ahf_result *out_host, int64_t *bound_idx_host,
                   int64_t cap);

/* Latency percentiles (microseconds from entering ahf_serve_submit until the
 * result is visible to ahf_serve_poll, nearest rank over the requests
 * completed since creation or the last reset) and throughput (completed
 * requests per second between the first submission and the last completion).
 * Any pointer may be NULL.  Errors: AHF_ERR_INVALID. */
int ahf_serve_stats(ahf_serve *s, double *p50_us, double *p99_us, double *throughput);

/* Counters since creation or the last reset; any pointer may be NULL:
 * requests accepted, completed, refused with AHF_ERR_FULL, batches run. */
int ahf_serve_counters(ahf_serve *s, int64_t *submitted, int64_t *completed, int64_t *rejected,
                       int64_t *batches);

/* Clear the latency samples and counters (requests in flight still count when
 * they complete). */
int ahf_serve_reset_stats(ahf_serve *s);

/* Stop accepting requests, finish every accepted one, stop the worker and
 * release the instance (results not yet polled are dropped).  NULL is
 * accepted. */
int ahf_serve_destroy(ahf_serve *s);

#ifdef __cplusplus
}
#endif
#endif /* AHF_H */
