// arc_internal.cuh -- device-side data layout and helpers shared by the libarc
// translation units (tracer, chemistry, host API).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "arc.h"

namespace arc {

// ---------------------------------------------------------------------------
// Units.  Photon rates on the device are carried in units of PHOT_UNIT
// photons/s so that rays of sources from 1e30 to 1e55 photons/s stay inside
// the normal FP32 range at every HEALPix level (a level-15 ray of a 1e47
// source carries ~8e-4 units, one of a 1e51 source at level 1 ~2e9 units).
// ---------------------------------------------------------------------------
constexpr double PHOT_UNIT = 1e40;
constexpr double EV_ERG = 1.602176634e-12;
constexpr double K_BOLTZ = 1.380649e-16;

// Status bits of the device status word.
enum : uint32_t {
    ERR_TIMEOUT = 1u << 0,    // an idle warp waited past its bound
    ERR_QUEUE_FULL = 1u << 1, // the global work queue could not take an entry
    ERR_RECORDS = 1u << 2,    // the ray record buffer overflowed
    ERR_SUBSTEP = 1u << 3,    // a chemistry cell hit the sub-step cap
    ERR_CAS_SPIN = 1u << 4,   // a queue CAS loop exceeded its bound
    ERR_FIELDS = 1u << 5,     // invalid gas field value found on the device
};

// ---------------------------------------------------------------------------
// Internal cell layout: 8x8x8 bricks, bricks in C order over ceil(n/8)^3,
// cells inside a brick in Morton order (k bit first).  A ray crossing a brick
// touches a handful of 128-byte lines instead of one line per cell as in the
// C-order layout, which raises L2 reuse of the absorber and accumulator
// records.  User-facing arrays stay in C order; the prep and finalize passes
// convert.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint32_t spread3(uint32_t v) {
    // three bits b2 b1 b0 -> b2 0 0 b1 0 0 b0
    return (v & 1u) | ((v & 2u) << 2) | ((v & 4u) << 4);
}
__host__ __device__ __forceinline__ uint64_t brick_index(int i, int j, int k, int nb) {
    const uint64_t b = ((uint64_t)(i >> 3) * nb + (uint64_t)(j >> 3)) * nb + (uint64_t)(k >> 3);
    const uint32_t m = spread3((uint32_t)k & 7u) | (spread3((uint32_t)j & 7u) << 1) |
                       (spread3((uint32_t)i & 7u) << 2);
    return (b << 9) | m;
}
__host__ __device__ __forceinline__ uint32_t compact3(uint32_t m) {
    return (m & 1u) | ((m >> 2) & 2u) | ((m >> 4) & 4u);
}

// ---------------------------------------------------------------------------
// Ray work item: the not-yet-traced children k_next..3 of one split (or the
// 4 pixels pixbase..pixbase+3 of an emitted group).  32 bytes, one sector.
// key bits: 0..47 pixbase (4 x parent pixel), 48..55 level, 56..58 k_next.
// ---------------------------------------------------------------------------
struct __align__(16) Entry {
    uint64_t key;
    uint32_t src;
    float r;        // start radius of the children [cells]
    float4 N;       // photons per child per group [PHOT_UNIT]
};
static_assert(sizeof(Entry) == 32, "entry is one 32-byte sector");

__host__ __device__ __forceinline__ uint64_t make_key(uint64_t pixbase, int level, int k) {
    return pixbase | ((uint64_t)level << 48) | ((uint64_t)k << 56);
}
__host__ __device__ __forceinline__ uint64_t key_pixbase(uint64_t key) { return key & 0xFFFFFFFFFFFFull; }
__host__ __device__ __forceinline__ int key_level(uint64_t key) { return (int)((key >> 48) & 0xFF); }
__host__ __device__ __forceinline__ int key_k(uint64_t key) { return (int)((key >> 56) & 0x7); }

// Per-source record on the device (sources sorted by luminosity, brightest first).
// The position is an unevaluated pair per axis, hi + lo: the caller's FP64
// value to ~1e-12 cell (hi alone would move the source by up to 3e-5 cell at
// 512 cells, which changes the photons sent through optically thick cells by
// ~1e-4).
struct __align__(16) SourceDev {
    float4 pos_thr;   // x, y, z [cells] (high parts), photon threshold of one l_base ray [PHOT_UNIT]
    float4 N0;        // photons of one l_base ray per group [PHOT_UNIT]
    float4 pos_lo;    // x, y, z low parts [cells]; w: group-0 photons of one l_base ray after
                      // optical depth 0.1 (N0.x exp(-0.1)), the optically thin radius test (Sec. 2.6)
    uint32_t id;      // index in the order the caller added the sources
    uint32_t pad[3];
};
static_assert(sizeof(SourceDev) == 64, "source record: two 32-byte sectors");
// Brick-cell indices are 32-bit: n <= ARC_MAX_N keeps ceil(n/8)^3 * 512 below 2^32.
#define ARC_MAX_N 1280

// Arguments of the tracer kernels.
struct TraceArgs {
    int n, nb, ng, l_base, l_max;
    uint32_t bstride_x, bstride_y;     // record-index step of one brick along x (512 nb^2) and y (512 nb)
    // cell records [2 * brick cells]: [2q] optical depth per cell length per
    // group, [2q + 1] photons absorbed per group (FP32 sums); kappa and acc
    // both point at the record array
    const float4* kappa;
    float4* acc;
    const SourceDev* src;
    int nsrc;
    float rsplit[ARC_MAX_LEVEL + 1];   // split distance per level [cells]
    float pixw[ARC_MAX_LEVEL + 1];     // pixel width per unit distance, sqrt(Omega_l)
    // sin and cos of pi j / 64, j = -16..16, as FP32 pairs (sin hi, sin lo, cos hi,
    // cos lo), formed once on the host in FP64 (fill_sincos_table)
    float4 sincos[33];
    int geo_corr;                      // geometric correction (Sec. 2.5) on
    // anisotropic escape (Sec. 2.2): open[src * nbase + pix] == 0 blocks emitted
    // ray pix of device source src (nullptr: all open)
    const uint8_t* open;
    int nbase;                         // rays emitted per source, 12 * 4^l_base
    // optically thin approximation (Sec. 2.6, extended kernels only): per
    // device source, the minimum over its rays of the length while the group-0
    // optical depth is below 0.1, as float bits (atomicMin)
    float* rnext;
    double* thin;                      // photons deposited by the thin fill [PHOT_UNIT]
    // emitted work: static array consumed by ticket
    const Entry* seeds;
    int nseeds;
    unsigned int* seed_head;
    // dynamic work queue (bounded MPMC ring, per-slot sequence numbers)
    Entry* qdata;
    unsigned long long* qseq;
    unsigned long long* qhead;
    unsigned long long* qtail;
    unsigned long long qmask;
    // bookkeeping
    long long* live;          // rays not yet finished (approximate until quiescence)
    int* n_idle;              // warps waiting for work
    unsigned int* status;     // device status word (ERR_*)
    unsigned int* heartbeat;  // progress counter for the idle-wait bound
    double* escaped;          // photons that left the box [PHOT_UNIT]
    double* rounding;         // photons the FP32 cell sums rounded away [PHOT_UNIT]
    unsigned long long* counters;  // segments, rays, splits, terminated, escaped, donations, maxlevel
    arc_ray_rec* recs;
    unsigned long long* nrec;
    unsigned long long rec_cap;
    int stack_log2;           // local work stack entries per warp = 1 << stack_log2
    unsigned long long idle_timeout_ns;
};

enum { CNT_SEG = 0, CNT_RAYS, CNT_SPLIT, CNT_TERM, CNT_ESC, CNT_DONATE, CNT_MAXLEVEL, CNT_N };
// counters[CNT_N] and [CNT_N + 1] (segments and traces over the context's life)
// follow the per-trace counters and are never reset
enum { CNT_SEG_TOTAL = CNT_N, CNT_TRACES_TOTAL, CNT_ALL };

// Launch wrappers (defined in arc_trace.cu / arc_chem.cu).
struct PrepArgs {
    int n, nb, ng;
    const float* nH;
    const float* xHI;
    const float* xHeI;
    const float* xHeII;
    float y;                  // n_He / n_H
    float sig_dx[3][ARC_MAX_GROUPS];   // sigma_{s,b} * dx [cm^3]: kappa = sum_s sig_dx n_s
    float4* rec;              // cell records (optical depth, absorbed photons)
};
struct FinalizeArgs {
    int n, nb, ng;
    const float* nH;
    const float* xHI;
    const float* xHeI;
    const float* xHeII;
    float y;
    float sig[3][ARC_MAX_GROUPS];      // sigma_{s,b} [cm^2]
    float egap_erg[3][ARC_MAX_GROUPS]; // (E_b - E_s) [erg]
    float scale;              // PHOT_UNIT / V [1/(s cm^3)]
    const float4* rec;        // cell records: absorbed photons at [2q + 1]
    float* gamma;             // 3*n^3
    float* heat;              // 3*n^3
    double* absorbed_part;    // per block FP64 partial of absorbed photons [PHOT_UNIT]
};
struct ChemArgs {
    long long ncell;
    float* nH;
    float* xHI;
    float* xHeI;
    float* xHeII;
    float* T;
    const float* gamma;
    const float* heat;
    double dt;
    float y, eps, xfloor, alpha_fixed, tcmb, compton_coef;
    int isothermal, coll_ion, compton;
    unsigned int* status;
    unsigned long long* counters;  // substeps, fp64 substeps, capped, surrogate-accepted cells (4)
    // optional list of cells to update (the surrogate's fallback list)
    const unsigned* list;
    const unsigned* list_count;
};

// ---------------------------------------------------------------------------
// Chemistry surrogate: per-cell MLP 12 -> 64 -> 64 -> 64 -> 4, SiLU, BF16
// weights, FP32 accumulation.  Features (before normalisation):
//   log10 nH, logit10 x_HI, logit10 x_HeI, logit10 x_HeII, log10 T,
//   log10(Gamma_s + 1e-30) x3, log10(H_s + 1e-37) x3, log10 dt,
// with logit10 x = log10(max(x, 1e-8) / max(1 - x, 1e-8)), which resolves
// fractions near 0 and near 1 alike.
// The network corrects a physics predictor (p0..p2, pT: the rate equations
// integrated exactly with the coefficients frozen at the start state, and
// the energy from trapezoidal heating minus the start cooling).  Targets
// (before normalisation): x_HI' - p0, x_HeI' - p1/y, x_HeII' - p2/y,
// log10(T'/pT).
// Flat FP32 parameter order: W1[64][12], b1[64], W2[64][64], b2[64],
// W3[64][64], b3[64], W4[4][64], b4[4]  (MLP_NPARAMS floats).
// The normalised FP32 features enter the first layer as two BF16 k-tiles,
// v = hi + lo with hi = bf16(v), lo = bf16(v - hi), both multiplied by the
// same BF16 W1: the inputs keep ~16 bits of precision at the cost of one
// more 16-wide MMA k-step.
// ---------------------------------------------------------------------------
constexpr int MLP_IN = 12, MLP_H = 64, MLP_OUT = 4;
constexpr int MLP_NPARAMS = MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H) + MLP_OUT * MLP_H + MLP_OUT;
static_assert(MLP_NPARAMS == ARC_MLP_NPARAMS, "surrogate parameter count");
static_assert(ARC_MLP_NNORM == 2 * MLP_IN + 3 * MLP_OUT, "surrogate normalisation block");
// padded bf16 row strides (rows land on distinct shared-memory banks)
constexpr int MLP_LD1 = 40, MLP_LDH = 72;
struct MlpDev {
    unsigned short W1[MLP_H * MLP_LD1];       // bf16 bits: [W1 | 0 0 0 0 | W1 | 0 0 0 0 | pad 8]
    unsigned short W2[MLP_H * MLP_LDH];
    unsigned short W3[MLP_H * MLP_LDH];
    unsigned short W4[8 * MLP_LDH];           // rows 4..7 zero
    float b1[MLP_H], b2[MLP_H], b3[MLP_H], b4[8];
    float in_mu[MLP_IN], in_sd[MLP_IN], out_mu[MLP_OUT], out_sd[MLP_OUT], out_s[MLP_OUT];
};
static_assert(sizeof(MlpDev) % 16 == 0, "MlpDev is copied to shared memory in 16-byte words");

// Surrogate features use the hardware base-2 logarithm (absolute error
// ~1e-7 in log10, below the ~2^-16 relative resolution the split BF16
// inputs keep).
__device__ __forceinline__ float flog10(float x) { return __log2f(x) * 0.30102999566398120f; }
__device__ __forceinline__ float logit10(float x) {
    return flog10(__fdividef(fmaxf(x, 1e-8f), fmaxf(1.0f - x, 1e-8f)));
}
// Surrogate features of one cell, in the order of the public header.
__device__ __forceinline__ void mlp_features(float nH, float xHI, float xHeI, float xHeII, float T,
                                             const float (&G)[3], const float (&H)[3], float ldt,
                                             float (&f)[MLP_IN]) {
    f[0] = flog10(fmaxf(nH, 1e-30f));
    f[1] = logit10(xHI);
    f[2] = logit10(xHeI);
    f[3] = logit10(xHeII);
    f[4] = flog10(T);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        f[5 + q] = flog10(G[q] + 1e-30f);
        f[8 + q] = flog10(H[q] + 1e-37f);
    }
    f[11] = ldt;
}
// Step change r_k from the network's k-th normalised output o.
__device__ __forceinline__ float mlp_change(const MlpDev& w, int k, float o) {
    return w.out_s[k] * sinhf(o * w.out_sd[k] + w.out_mu[k]);
}
struct SurrogateArgs {
    const MlpDev* w;
    float tol_x, tol_e;        // residual-check tolerances (abundance, relative energy)
    float gate;                // cells the plain solver handles in <= gate sub-steps skip the network
    unsigned* fb_list;         // cells that failed the check (for the plain solver)
    unsigned* fb_count;
};
cudaError_t launch_chem_surrogate(const ChemArgs& c, const SurrogateArgs& s, cudaStream_t st);
cudaError_t launch_pack_mlp(const float* params, const float* norm, MlpDev* out, cudaStream_t s);
cudaError_t launch_mlp_eval(const MlpDev* w, const float* X, long long n, float* Y, cudaStream_t s);
cudaError_t launch_mlp_targets(const ChemArgs& c, const float* x1, const float* T1, float* Y, cudaStream_t s);

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s);
cudaError_t launch_seed_reset(const TraceArgs& a, unsigned long long qcap, int nseeds, cudaStream_t s);
cudaError_t launch_trace(const TraceArgs& a, int grid, int block, cudaStream_t s);
// the HEALPix longitude table of TraceArgs (host)
void fill_sincos_table(TraceArgs& a);
cudaError_t launch_finalize(const FinalizeArgs& a, int blocks, cudaStream_t s);
cudaError_t launch_budget(const double* part, int nparts, const double* escaped, const double* rounding,
                          const double* thin, double* out,
                          cudaStream_t s);
cudaError_t launch_validate(const float* nH, const float* xHI, const float* xHeI,
                            const float* xHeII, const float* T, long long ncell,
                            unsigned int* status, cudaStream_t s);
// Optically thin approximation (Sec. 2.6): seeds start at rthin of their
// source and rnext is reset (begin); cells within rthin of a source take the
// thin-limit absorption (fill); rthin takes the radii the trace measured
// (commit).  All arrays are per device source.
struct ThinFillArgs {
    int n, nb, nsrc;
    const SourceDev* src;
    const float* rthin;
    float nbase;              // rays per source: S_b = N0_b * nbase
    float4* rec;
    double* thin;             // ledger of the fill's photons [PHOT_UNIT]
    double* rounding;         // rounding ledger of the FP32 cell sums
};
cudaError_t launch_thin_begin(Entry* seeds, int nseeds, const float* rthin, float* rnext, int nsrc,
                              cudaStream_t s);
cudaError_t launch_thin_fill(const ThinFillArgs& a, cudaStream_t s);
cudaError_t launch_thin_commit(float* rthin, const float* rnext, int nsrc, cudaStream_t s);
cudaError_t launch_make_seeds(const SourceDev* src, int nsrc, int l_base, Entry* seeds,
                              cudaStream_t s);
cudaError_t launch_chem(const ChemArgs& a, cudaStream_t s);
cudaError_t launch_rt_timestep(const ChemArgs& c, float sigd, float eps, unsigned* out, cudaStream_t s);
int trace_smem_bytes(int block, int stack_log2);
// rec: the per-ray-record variant; ext: the variant with emission masks and
// the optically thin radius
const void* trace_kernel_ptr(int ng, bool rec = false, bool ext = false);

}  // namespace arc
