/*
 * arc.h -- C ABI of libarc, a single-GPU (sm_103a) implementation of the hot
 * path of ARC, the photon-conserving adaptive ray tracer of Hartley & Ricotti
 * (arXiv 1807.07094): per-source HEALPix ray tracing with photon-conserving
 * multi-frequency absorption, and the per-cell H/He ionisation and thermal
 * update that consumes its rates.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units      CGS.  Positions are in grid units: cell (i,j,k) spans
 *            [i,i+1) x [j,j+1) x [k,k+1); coordinate x maps to index i.
 * Layout     Every per-cell array is FP32, C order [i][j][k] (k fastest),
 *            n^3 elements; per-species arrays are species-major
 *            [s][i][j][k] with s = 0 HI, 1 HeI, 2 HeII.
 * Ownership  The context owns every device buffer it allocates; inputs are
 *            copied in.  Pointers returned by arc_trace stay valid until the
 *            next arc_trace or arc_destroy.
 * Streams    All work is queued on the stream given to arc_create (NULL: the
 *            context creates and owns a non-blocking stream).  Only the calls
 *            documented as synchronising wait for the GPU; device outputs are
 *            written on that stream, so a caller reading them on another
 *            stream must synchronise first.
 * Errors     Every call returns an arc_status.  Errors found by a kernel
 *            (queue overflow, a bounded wait that gave up, a chemistry cell
 *            that hit the sub-step cap) are recorded in a device status word
 *            and returned by the next synchronising call.  arc_last_error()
 *            gives a one-line text for the most recent failure.
 * Threads    A context must not be used by two host threads at once.
 */
#ifndef ARC_H
#define ARC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ARC_MAX_GROUPS 4    /* frequency groups carried per ray */
#define ARC_MAX_LEVEL 15    /* deepest HEALPix level a ray may reach */

typedef enum {
    ARC_OK = 0,
    ARC_E_INVALID = 1,   /* bad argument or input field value                       */
    ARC_E_OOM = 2,       /* device allocation failed                                */
    ARC_E_CUDA = 3,      /* a CUDA runtime call failed                              */
    ARC_E_TIMEOUT = 4,   /* a bounded wait in the persistent tracer gave up         */
    ARC_E_BUDGET = 5,    /* photon budget failed to close within 1e-9               */
    ARC_E_STATE = 6,     /* call out of order (e.g. trace before fields are set)    */
    ARC_E_OVERFLOW = 7,  /* ray work queue or record buffer capacity exceeded       */
    ARC_E_SUBSTEP = 8    /* a chemistry cell hit the sub-step cap                   */
} arc_status;

typedef struct arc_ctx arc_ctx;

/* Uniform cubic grid of n^3 cells and physical side box_cm (Sec. 2.3). */
typedef struct {
    int n;               /* cells per side, 1 .. 1280 (32-bit cell-record index)    */
    double box_cm;       /* side length [cm]                                        */
} arc_grid;

/*
 * Method parameters.  Frequency groups (Sec. 2.2): each group b is one
 * frequency with photon energy E_group_eV[b] and cross sections sigma[s][b]
 * [cm^2] for s = HI, HeI, HeII.  The defaults used by the workloads are in
 * the comments.
 */
typedef struct {
    int ngroups;                          /* 1 .. ARC_MAX_GROUPS                        */
    double E_group_eV[ARC_MAX_GROUPS];    /* mean photon energy per group [eV]          */
    double sigma[3][ARC_MAX_GROUPS];      /* sigma_{s,b} [cm^2]                         */
    double Y;                             /* helium mass fraction (0.24; 0 = pure H)    */
    double phi;                           /* split when fewer than phi rays cross a
                                             cell face (4)  -- Sec. 2.4, Fig. 1         */
    int l_base;                           /* HEALPix level of emitted packets (1)       */
    int l_max;                            /* deepest level; l_max rays never split (14) */
    double term_frac;                     /* terminate a ray below this fraction of its
                                             share of the emission (1e-6)              */
    double eps_sub;                       /* sub-cycle fractional-change limit (0.1)
                                             -- Sec. 2.7                               */
    double x_fp64;                        /* cells with x_HI below this take their
                                             species update in FP64 (1e-4); also the
                                             floor of the step limiter                 */
    int isothermal;                       /* 1: temperature fixed                      */
    double alpha_B_fixed;                 /* > 0: constant case-B alpha_HII [cm^3/s]   */
    int coll_ion;                         /* 1: collisional ionisation on              */
    double z_compton;                     /* >= 0: Compton cooling off the CMB at z    */
    int geo_correction;                   /* 1: geometric correction (Sec. 2.5, Eqs.
                                             correction, correction2): when a segment's
                                             midpoint is within half a pixel width
                                             L = r sqrt(Omega_l) of the nearest cell
                                             face, 1 - f_c (f_c = 1/2 + D_edge / L) of
                                             its absorbed photons go to the neighbour
                                             across that face; 0: off                  */
    int thin_approx;                      /* 1: optically thin approximation (Sec. 2.6):
                                             every source carries a radius R (0 at
                                             first); cells whose centre lies within R
                                             take the thin limit of Eq. (ion),
                                             S_b sigma_{s,b} / (4 pi r^2) per absorber
                                             (r from the source to the cell centre,
                                             at least half a cell), rays start at
                                             distance R, and each trace sets the next
                                             R to the minimum over the source's rays of
                                             the length while the optical depth of
                                             group 0 (which must be the softest) is
                                             below 0.1; 0: off                         */
} arc_params;

/* Counters of the last arc_trace / arc_chem_update (arc_stats synchronises). */
typedef struct {
    uint64_t segments;       /* ray-cell segments traced                              */
    uint64_t rays;           /* rays traced (every node of every ray tree)            */
    uint64_t splits;         /* rays that split into four children                    */
    uint64_t terminated;     /* rays stopped by the photon threshold                  */
    uint64_t escaped_rays;   /* rays that left the box                                */
    uint64_t donations;      /* work items moved to the global queue                  */
    uint32_t max_level;      /* deepest HEALPix level reached                         */
    uint32_t error_word;     /* raw device status bits of the last trace/chemistry    */
    uint64_t chem_substeps;  /* sub-steps summed over cells                           */
    uint64_t chem_fp64_substeps; /* sub-steps taken on the FP64 branch                */
    uint64_t chem_capped;    /* cells that hit the sub-step cap                       */
    double trace_ms;         /* device time of the last trace (events)                */
    double chem_ms;          /* device time of the last chemistry update              */
    uint64_t segments_total; /* segments summed over every trace of this context      */
    uint64_t traces_total;   /* traces run by this context                            */
    uint64_t surrogate_cells;/* cells updated by the surrogate in the last chemistry  */
    uint64_t fallback_cells; /* cells the residual check sent to the plain solver     */
} arc_stats_t;

/* One record per ray (test aid, see arc_set_records). */
typedef struct {
    uint32_t src;            /* source index in the order sources were added           */
    uint8_t level;           /* HEALPix level                                          */
    uint8_t end;             /* 1 split, 2 escaped, 3 terminated, 4 blocked by the
                                source's emission mask (no photons, no cells)         */
    uint16_t pad;
    uint64_t pix;            /* nested pixel index at that level                       */
    uint32_t visits;         /* cell segments traced, zero-length ones included; 0 for
                                a ray that starts at or beyond its split distance
                                (thin_approx) and splits at once                     */
    float r1;                /* distance from the source where the ray ended [cells]  */
} arc_ray_rec;

/*
 * arc_create -- allocate a context for an n^3 grid (Sec. 2.3).
 *   out      receives the context (set to NULL on failure)
 *   g, p     grid and parameters, copied
 *   stream   cudaStream_t to queue all work on (NULL: a private stream)
 * Allocates the field, rate, accumulator and work-queue buffers on the
 * current device.  Returns ARC_E_INVALID for out-of-range parameters,
 * ARC_E_OOM if an allocation fails.
 */
arc_status arc_create(arc_ctx** out, const arc_grid* g, const arc_params* p, void* stream);

/*
 * arc_set_fields -- copy in the gas state (Sec. 2.3): hydrogen number density
 * nH [cm^-3], neutral fractions x_HI = n_HI/n_H, x_HeI = n_HeI/n_He, singly
 * ionised fraction x_HeII = n_HeII/n_He (n_He = Y/(4(1-Y)) n_H), temperature
 * T [K].  n^3 FP32 each, C order; on_device = 1 for device pointers, 0 for
 * host pointers.  Validates: finite values, nH >= 0, fractions in [0,1],
 * x_HeI + x_HeII <= 1, T > 0; returns ARC_E_INVALID otherwise (the context's
 * fields are then unspecified).  Synchronises.
 */
arc_status arc_set_fields(arc_ctx* ctx, const float* nH, const float* xHI, const float* xHeI,
                          const float* xHeII, const float* T, int on_device);

/*
 * arc_add_sources -- append point sources (Sec. 2.1, 2.4).
 *   pos   nsrc*3 host doubles, grid units, inside [0,n)^3
 *   ndot  nsrc*ngroups host doubles, photons/s emitted in each group
 * Each source emits 12*4^l_base rays sharing its output equally (Sec. 2.4).
 * Positions are kept on the device as FP32 pairs (hi + lo, ~1e-12 cell), so
 * rays start from the caller's FP64 position; sources with no emission are
 * kept but trace no rays.  Returns ARC_E_INVALID for a position outside the
 * box or a negative/NaN rate.
 */
arc_status arc_add_sources(arc_ctx* ctx, int nsrc, const double* pos, const double* ndot);

/* arc_clear_sources -- remove all sources. */
arc_status arc_clear_sources(arc_ctx* ctx);

/*
 * arc_trace -- one radiative-transfer pass over all sources (Sec. 2.1 steps
 * i and iii; Sec. 2.4 Eq. ion; Sec. 2.8 photoheating).
 *   dt      time step [s]; only scales the photon counts in budget
 *   gamma   receives a device pointer to 3*n^3 photoionisation rates per
 *           absorber [1/s] (species-major, C order); may be NULL
 *   heat    receives a device pointer to 3*n^3 photoheating rates per
 *           absorber [erg/s]; may be NULL
 *   budget  NULL, or host double[4] receiving photons over dt:
 *           [0] launched into rays, [1] absorbed in cells from the rays, [2]
 *           escaped from the box, [3] emitted by the sources (FP64 input sum).
 *           [0] differs from [3] by the FP32 rounding of each ray's initial
 *           share and by the rays an emission mask blocks.  The photons of the
 *           thin fill (thin_approx) are in no entry: see arc_get_thin_radii.
 * With budget != NULL the call synchronises and returns ARC_E_BUDGET if
 * |launched - absorbed - escaped| > 1e-9 launched, ARC_E_TIMEOUT or
 * ARC_E_OVERFLOW if the tracer recorded such an error.
 */
arc_status arc_trace(arc_ctx* ctx, double dt, float** gamma, float** heat, double* budget);

/*
 * arc_chem_update -- advance the gas state by dt [s] with the rates of the
 * last arc_trace held constant (Sec. 2.7 Eqs. diffeq and anninos, sub-cycled;
 * Sec. 2.8 heating and cooling).  Asynchronous.  Cells whose x_HI is below
 * x_fp64 take their species update in FP64.
 */
arc_status arc_chem_update(arc_ctx* ctx, double dt);

/*
 * arc_step -- arc_trace followed by arc_chem_update, replayed from a CUDA
 * graph captured on the first call (and re-captured when dt or the sources
 * change).  Asynchronous.
 */
arc_status arc_step(arc_ctx* ctx, double dt);

/*
 * arc_get_fields -- copy out x_HI, x_HeI, x_HeII, T (n^3 FP32 each, C order)
 * to device (on_device = 1) or host memory; any pointer may be NULL.
 * Synchronises.
 */
arc_status arc_get_fields(arc_ctx* ctx, float* xHI, float* xHeI, float* xHeII, float* T,
                          int on_device);

/*
 * arc_set_records -- test aid: when buf (device memory of cap arc_ray_rec)
 * is not NULL, the next traces write one record per ray; the count is
 * returned by arc_get_record_count.  Records cost a global atomic per ray.
 */
arc_status arc_set_records(arc_ctx* ctx, void* buf, int64_t cap);
arc_status arc_get_record_count(arc_ctx* ctx, int64_t* count);

/* arc_stats -- counters of the last trace and chemistry update.  Synchronises. */
arc_status arc_stats(arc_ctx* ctx, arc_stats_t* out);

/*
 * arc_set_tuning -- launch shape of the persistent tracer: threads per block
 * (multiple of 32, 64..256), blocks per SM (0 = occupancy limit) and local
 * work-stack entries per warp (power of two, 64..256).  0 keeps a value.
 */
arc_status arc_set_tuning(arc_ctx* ctx, int block_threads, int blocks_per_sm, int stack_entries);
/* arc_get_tuning -- the launch shape in use (any pointer may be NULL). */
arc_status arc_get_tuning(arc_ctx* ctx, int* block_threads, int* blocks_per_sm, int* stack_entries);

/*
 * arc_trace_noalloc -- one radiative-transfer pass, like arc_trace, that
 * allocates nothing.  The paper has no counterpart: it is a deployment variant
 * of the tracer for callers that cannot allocate device memory when they need
 * a trace.  Simulation codes that embed a radiative-transfer step often hand
 * all of the GPU's memory to their own pool allocator at start-up (to avoid
 * fragmentation and late out-of-memory failures in runs of days), so a library
 * that asks the driver for more finds nothing left or is forbidden to ask; and
 * cudaFree waits for all work on the device, which such codes cannot afford
 * inside their time-step loop.  arc_create allocates its buffers, so these
 * callers use this entry point instead.
 *
 *   g, p            grid and parameters as for arc_create; n <= ARC_NOALLOC_MAX_N,
 *                   l_base <= 2, no optically thin approximation
 *   nH..xHeII       device pointers, n^3 FP32 each, C order (as arc_set_fields)
 *   nsrc, pos, ndot host arrays as for arc_add_sources (pos nsrc*3, ndot
 *                   nsrc*ngroups), nsrc <= ARC_NOALLOC_MAX_SOURCES
 *   gamma, heat     caller-owned device buffers of 3 n^3 FP32 each (outputs, as
 *                   returned by arc_trace)
 *   budget          NULL or host double[4], as for arc_trace
 *   stream          cudaStream_t for the work (NULL = legacy default stream)
 *
 * Scratch memory is one fixed file-scope device array of about 18 MB that every
 * device which loads libarc holds until the process exits; the call makes no
 * cudaMalloc, cudaFree or other allocating call.  The first call on a device
 * looks up that array's device address (cudaGetSymbolAddress) with the device
 * current.  All calls share the array and it keeps the last call's contents
 * (each call clears what must start at zero), so calls whose GPU work overlaps
 * -- on different streams or from different host threads -- race and corrupt
 * each other's results.  The call copies the source table from host memory and
 * waits for the stream before it returns.  Returns ARC_E_INVALID for sizes
 * beyond the maximum or bad arguments, and the tracer errors of arc_trace
 * (ARC_E_TIMEOUT, ARC_E_OVERFLOW, ARC_E_BUDGET); the binding must check the
 * array sizes, which the C interface cannot see.
 */
#define ARC_NOALLOC_MAX_N 64
#define ARC_NOALLOC_MAX_SOURCES 256
arc_status arc_trace_noalloc(const arc_grid* g, const arc_params* p, const float* nH,
                             const float* xHI, const float* xHeI, const float* xHeII, int nsrc,
                             const double* pos, const double* ndot, float* gamma, float* heat,
                             double* budget, void* stream);

/*
 * arc_autotune -- choose the tracer's launch shape for the current fields and
 * sources by timing it: every candidate (threads per block 128/256, blocks per
 * SM from the occupancy limit down, deque entries per warp 64/128/256) traces
 * the brightest `max_sources` sources (0 = all) `reps` times on the context
 * stream; the fastest shape by CUDA-event time is kept (as arc_set_tuning).
 * Synchronises.  best_ms (may be NULL) receives the best trace time.
 * The rates left in the context's buffers afterwards are those of the last
 * candidate run: call arc_trace again before using them.
 */
arc_status arc_autotune(arc_ctx* ctx, int max_sources, int reps, double* best_ms);

/*
 * arc_rt_timestep -- radiative-transfer time step (Sec. 2.9) from the
 * context's current fields and the HI photoionisation rate of the last
 * arc_trace.  Per cell dn_HI/dt = alpha n_e n_HII - (Gamma_HI + beta n_e) n_HI
 * (Eq. anninos); *dt_n = min over cells with n_HI sigma d > 0.5 of
 * eps n_HI / |dn_HI/dt| ("minimum neutral fraction change"), *dt_I = min over
 * all cells of eps / (sigma d |dn_HI/dt|) ("minimum intensity change"); sigma
 * is the HI cross section of the first group, d the cell width; seconds,
 * +inf when no cell qualifies.  FP32 per cell.  Synchronises.
 */
arc_status arc_rt_timestep(arc_ctx* ctx, double eps, double* dt_n, double* dt_I);

/* ------------------------------------------------------------------------
 * Chemistry surrogate (a learned stand-in for the sub-cycled update of
 * arc_chem_update; the paper has none).  Per cell a physics predictor -- the
 * rate equations of Eq. (anninos) integrated exactly with the coefficients
 * frozen at the start state (HI: one exponential; He: the HeI/HeII chain as
 * a 2x2 linear system), and the energy from the trapezoidal heating of the
 * start and predicted abundances minus the start cooling -- is corrected by
 * an MLP 12 -> 64 -> 64 -> 64 -> 4 with SiLU that maps
 *   features  log10 nH, logit10 x_HI, logit10 x_HeI, logit10 x_HeII, log10 T,
 *             log10(Gamma_s + 1e-30) x3, log10(H_s + 1e-37) x3, log10 dt
 *   (logit10 x = log10(max(x, 1e-8) / max(1 - x, 1e-8)))
 * to the corrections r = (x_HI' - p_HI, x_HeI' - p_HeI, x_HeII' - p_HeII,
 * log10(T'/p_T)).  Inputs are normalised as (v - mu) / sd; the network's
 * k-th output o_k stands for r_k = s_k sinh(o_k sd_k + mu_k), so that small
 * and large corrections are resolved alike.
 * Parameters: ARC_MLP_NPARAMS FP32 values in the order
 *   W1[64][12], b1[64], W2[64][64], b2[64], W3[64][64], b3[64], W4[4][64], b4[4];
 * normalisation: 36 FP32 values  in_mu[12], in_sd[12], out_mu[4], out_sd[4],
 * out_s[4] (all sd and s > 0).
 * Products run on the tensor cores with BF16 operands and FP32 accumulation.
 * ------------------------------------------------------------------------ */
#define ARC_MLP_NPARAMS 9412
#define ARC_MLP_NNORM 36

/*
 * arc_set_surrogate -- load surrogate parameters (host arrays) into the
 * context and use them in arc_chem_update / arc_step.  Per cell the plain
 * solver's cost is estimated from the predictor's changes (its limiter
 * allows a fraction eps_sub of x_HI, x_HII and E per sub-step); cells
 * estimated at <= gate sub-steps are left to the plain solver.  The others
 * take the corrected prediction unless a residual check rejects it -- the
 * step re-integrated in two halves with the coefficients frozen at 1/4 and
 * 3/4 of the way from start to prediction must reproduce each predicted
 * abundance within tol_x (helium per He atom) and the predicted energy
 * within tol_e of the energy -- in which case the plain sub-cycled solver
 * updates that cell.  params = NULL switches the surrogate off.
 * tol_x, tol_e > 0, gate >= 0 (0: every cell tries the network).
 * Synchronises.
 */
arc_status arc_set_surrogate(arc_ctx* ctx, const float* params, const float* norm, double tol_x, double tol_e,
                             double gate);

/* Training.  A trainer holds FP32 master weights, AdamW moments and the
 * activations of one batch of up to max_batch samples (a multiple of 16). */
/*
 * arc_set_emission_mask -- anisotropic escape (Sec. 2.2): each source emits
 * its mean per-ray share on the open rays only and nothing on the others.
 *   open   nsrc * 12*4^l_base bytes, source-major in the order sources were
 *          added, ray index = nested HEALPix pixel at level l_base; nonzero =
 *          open.  NULL or count 0 removes the mask.
 *   count  number of bytes in open
 * Copied.  Adding or clearing sources removes the mask.  Returns
 * ARC_E_INVALID for a count that does not match the sources, or when
 * thin_approx is on (the two do not combine).
 */
arc_status arc_set_emission_mask(arc_ctx* ctx, const uint8_t* open, int64_t count);

/*
 * arc_set_thin_radii / arc_get_thin_radii -- the optically thin radius R of
 * each source (Sec. 2.6; thin_approx only, else ARC_E_STATE), in grid cells
 * and in the order sources were added.  A trace uses the current radii and
 * then replaces them with the ones it measured.  Adding or clearing sources
 * sets every radius to 0.  set: nsrc must equal the sources added, radii
 * in [0, 1e9] cells (ARC_E_INVALID otherwise); synchronises.  get: radii
 * (may be NULL) receives them; thin_photons (may be NULL) the photons the
 * thin fill deposited during the last trace, over its dt; synchronises.
 */
arc_status arc_set_thin_radii(arc_ctx* ctx, const double* radii, int nsrc);
arc_status arc_get_thin_radii(arc_ctx* ctx, double* radii, int nsrc, double* thin_photons);

/*
 * arc_set_fault -- failure-detection test aid.  live_bias > 0 adds that many
 * phantom unfinished rays to the tracer's count at the start of every trace,
 * so the count never reaches zero and the warps, once out of work, wait for
 * work that never comes; idle_timeout_s bounds that wait (default 10 s,
 * 1 ms .. 60 s).  When the bound runs out the tracer sets its timeout status
 * and returns; arc_trace then reports ARC_E_TIMEOUT (with a budget) and the
 * context stays usable.  live_bias 0 restores normal tracing.  Applies to
 * eager traces (arc_trace; the write uses a host value, not for capture).
 */
arc_status arc_set_fault(arc_ctx* ctx, int64_t live_bias, double idle_timeout_s);

typedef struct arc_mlp_trainer arc_mlp_trainer;
arc_status arc_mlp_trainer_create(arc_mlp_trainer** out, int max_batch, void* stream);
/* copy in parameters (host, ARC_MLP_NPARAMS) and reset the AdamW state */
arc_status arc_mlp_trainer_set_params(arc_mlp_trainer* t, const float* params);
arc_status arc_mlp_trainer_get_params(arc_mlp_trainer* t, float* params);
/* Gradient of the mean-squared error over n samples (n % 16 == 0, n <= max_batch).
 * X: device n x 12 normalised features; Y: device n x 4 normalised targets
 * ((asinh(r_k / s_k) - mu_k) / sd_k);
 * grad (host ARC_MLP_NPARAMS, may be NULL) and loss (host, may be NULL) receive
 * the result.  Synchronises. */
arc_status arc_mlp_grad(arc_mlp_trainer* t, const float* X, const float* Y, int n, float* grad, double* loss);
/* One AdamW step (beta1 0.9, beta2 0.999, decoupled weight decay wd on the
 * matrices).  loss (may be NULL) receives the batch loss before the step and
 * then the call synchronises; with loss = NULL it is asynchronous. */
arc_status arc_mlp_train_step(arc_mlp_trainer* t, const float* X, const float* Y, int n, double lr, double wd,
                              double* loss);
void arc_mlp_trainer_destroy(arc_mlp_trainer* t);
/* Inference kernel of arc_chem_update's surrogate on given raw features:
 * X device n x 12 (unnormalised), Y device n x 4 (the changes r_k).
 * Allocates its own weight buffers; synchronises. */
arc_status arc_mlp_eval(const float* params, const float* norm, const float* X, long long n, float* Y,
                        void* stream);

/* Surrogate features of n cells (device arrays of n FP32; gamma, heat 3 x n
 * species-major) -> X device n x 12, as the inference kernel forms them. */
arc_status arc_mlp_features(const float* nH, const float* xHI, const float* xHeI, const float* xHeII,
                            const float* T, const float* gamma, const float* heat, double dt, long long n, float* X,
                            void* stream);
/* Surrogate training targets on the context's chemistry switches: the
 * corrections of a step's end state (x1: 3 x n fractions HI, HeI, HeII; T1)
 * to the physics predictor started from (nH, x0: 3 x n, T0) with rates
 * gamma, heat (3 x n each) over dt -> Y n x 4 (device arrays).  Runs on the
 * context's stream and synchronises. */
arc_status arc_mlp_targets(arc_ctx* ctx, const float* nH, const float* x0, const float* T0, const float* gamma,
                           const float* heat, const float* x1, const float* T1, double dt, long long n, float* Y);

/* Text of the most recent error on this context (never NULL). */
const char* arc_last_error(const arc_ctx* ctx);

/* Release every buffer of the context.  NULL is ignored. */
void arc_destroy(arc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
