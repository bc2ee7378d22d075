// arc_noalloc.cu -- arc_trace_noalloc: one radiative-transfer pass that
// allocates nothing.
//
// Some callers cannot allocate device memory when they need a trace.
// Simulation codes that embed a radiative-transfer step commonly give the
// whole GPU memory to their own pool allocator when they start (so that a run
// of days neither fragments memory nor fails late for lack of it); a library
// that then asks the driver for memory finds none, or is not allowed to ask.
// Such codes also cannot let a library call cudaFree inside their time-step
// loop, since it waits for all work on the device.  For them this entry point
// runs the same tracer kernels as arc_trace, but every scratch buffer
// (optical-depth records and absorbed photons, work queue, source table,
// counters) lives in one file-scope device array of fixed size, so grids and
// source counts are capped (ARC_NOALLOC_MAX_N, ARC_NOALLOC_MAX_SOURCES).  The
// caller passes the gas fields and receives the rates in its own device
// buffers.
//
// The array is shared by every call in the process and keeps the last call's
// contents; each call clears what must start at zero.  Calls whose GPU work
// overlaps (different streams, or host threads racing) corrupt each other.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "arc_internal.cuh"

using namespace arc;

namespace {

constexpr int NA_MAX_N = ARC_NOALLOC_MAX_N;
constexpr int NA_MAX_SRC = ARC_NOALLOC_MAX_SOURCES;
constexpr int NA_MAX_LBASE = 2;
constexpr unsigned long long NA_QCAP = 1ull << 18;   // work-queue slots
constexpr int NA_NPARTS = 152 * 8;                    // FP64 partial sums of finalize
constexpr int NA_NB = (NA_MAX_N + 7) / 8;
constexpr size_t NA_CELLS = (size_t)NA_NB * NA_NB * NA_NB * 512;
constexpr int NA_MAX_SEEDS = NA_MAX_SRC * (3 << (2 * NA_MAX_LBASE));

struct NaScalars {
    unsigned long long qhead, qtail;
    long long live;
    int n_idle;
    unsigned int seed_head;
    unsigned int status;
    unsigned int heartbeat;
    double escaped;
    double rounding;
    unsigned long long counters[CNT_ALL];
    unsigned long long nrec;
    double budget_out[2];
};

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t OFF_REC = 0;   // cell records: optical depth, absorbed photons
constexpr size_t OFF_QDATA = al(OFF_REC + 2 * NA_CELLS * sizeof(float4));
constexpr size_t OFF_QSEQ = al(OFF_QDATA + NA_QCAP * sizeof(Entry));
constexpr size_t OFF_SEEDS = al(OFF_QSEQ + NA_QCAP * sizeof(unsigned long long));
constexpr size_t OFF_SRC = al(OFF_SEEDS + (size_t)NA_MAX_SEEDS * sizeof(Entry));
constexpr size_t OFF_PARTS = al(OFF_SRC + (size_t)NA_MAX_SRC * sizeof(SourceDev));
constexpr size_t OFF_SCAL = al(OFF_PARTS + NA_NPARTS * sizeof(double));
constexpr size_t NA_BYTES = al(OFF_SCAL + sizeof(NaScalars));

// The scratch: file scope, fixed size (about 18 MB), held by every device
// that loads the library until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// device address of the scratch per device, taken once with that device current
constexpr int NA_MAX_DEVICES = 64;
unsigned char* g_scratch_addr[NA_MAX_DEVICES] = {nullptr};

double na_r_split(double phi, int level) {
    const double omega = 4.0 * M_PI / (12.0 * pow(4.0, level));
    return 1.0 / sqrt(phi * omega);
}

}  // namespace

extern "C" arc_status arc_trace_noalloc(const arc_grid* g, const arc_params* p, const float* nH,
                                        const float* xHI, const float* xHeI, const float* xHeII,
                                        int nsrc, const double* pos, const double* ndot, float* gamma,
                                        float* heat, double* budget, void* stream_v) {
    if (!g || !p || !nH || !xHI || !xHeI || !xHeII || !gamma || !heat) return ARC_E_INVALID;
    if (g->n < 1 || g->n > NA_MAX_N || !(g->box_cm > 0)) return ARC_E_INVALID;
    if (nsrc < 0 || nsrc > NA_MAX_SRC || (nsrc > 0 && (!pos || !ndot))) return ARC_E_INVALID;
    if (p->thin_approx) return ARC_E_INVALID;   // needs per-source state across traces
    if (p->ngroups < 1 || p->ngroups > ARC_MAX_GROUPS || p->l_base < 1 || p->l_base > NA_MAX_LBASE ||
        p->l_max < p->l_base || p->l_max > ARC_MAX_LEVEL || !(p->phi > 0) ||
        !(p->term_frac > 0 && p->term_frac < 1) || !(p->Y >= 0 && p->Y < 1))
        return ARC_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream_v;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return ARC_E_CUDA;
    if (!g_scratch_addr[dev]) {
        // first call on this device: host code needs the array's device address
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return ARC_E_CUDA;
        g_scratch_addr[dev] = (unsigned char*)ptr;
    }
    unsigned char* base = g_scratch_addr[dev];
    float4* rec = (float4*)(base + OFF_REC);
    Entry* qdata = (Entry*)(base + OFF_QDATA);
    unsigned long long* qseq = (unsigned long long*)(base + OFF_QSEQ);
    Entry* seeds = (Entry*)(base + OFF_SEEDS);
    SourceDev* dsrc = (SourceDev*)(base + OFF_SRC);
    double* parts = (double*)(base + OFF_PARTS);
    NaScalars* scal = (NaScalars*)(base + OFF_SCAL);

    const int n = g->n, nb = (n + 7) / 8, G = p->ngroups;
    const double dx = g->box_cm / n;
    const double y = p->Y / (4.0 * (1.0 - p->Y));

    // source table on the host stack, brightest first (insertion sort by index)
    SourceDev hsrc[NA_MAX_SRC];
    int order[NA_MAX_SRC];
    double total[NA_MAX_SRC];
    int ns = 0;
    const double nrays = 12.0 * pow(4.0, p->l_base);
    double launched = 0.0, emitted = 0.0;
    for (int i = 0; i < nsrc; ++i) {
        double t = 0.0;
        for (int a = 0; a < 3; ++a)
            if (!(pos[3 * i + a] >= 0.0 && pos[3 * i + a] < (double)n)) return ARC_E_INVALID;
        for (int b = 0; b < G; ++b) {
            const double v = ndot[(size_t)i * G + b];
            if (!(v >= 0.0) || !isfinite(v)) return ARC_E_INVALID;
            t += v;
        }
        if (t > 0.0) {
            total[i] = t;
            int k = ns++;
            while (k > 0 && total[order[k - 1]] < t) {
                order[k] = order[k - 1];
                --k;
            }
            order[k] = i;
        }
    }
    for (int k = 0; k < ns; ++k) {
        const int i = order[k];
        float N0[ARC_MAX_GROUPS] = {0.f, 0.f, 0.f, 0.f};
        double tot = 0.0;
        for (int b = 0; b < G; ++b) {
            N0[b] = (float)(ndot[(size_t)i * G + b] / PHOT_UNIT / nrays);
            launched += (double)N0[b] * nrays * PHOT_UNIT;
            tot += (double)N0[b];
        }
        emitted += total[i];
        float ph[3], pl[3];
        for (int a = 0; a < 3; ++a) {   // the FP64 position as an FP32 pair
            ph[a] = (float)pos[3 * i + a];
            pl[a] = (float)(pos[3 * i + a] - (double)ph[a]);
        }
        hsrc[k].pos_thr = make_float4(ph[0], ph[1], ph[2], (float)(p->term_frac * tot));
        hsrc[k].N0 = make_float4(N0[0], N0[1], N0[2], N0[3]);
        hsrc[k].pos_lo = make_float4(pl[0], pl[1], pl[2], 0.f);   // no optically thin radius on this path
        hsrc[k].id = (uint32_t)i;
        hsrc[k].pad[0] = hsrc[k].pad[1] = hsrc[k].pad[2] = 0;
    }
    const int per_src = 3 << (2 * p->l_base);
    const int nseeds = ns * per_src;

#define NA_CK(call)                          \
    do {                                     \
        if ((call) != cudaSuccess) return ARC_E_CUDA; \
    } while (0)

    // everything that must start at zero is cleared here: the scalars; the
    // accumulators are zeroed by the prep kernel, the queue by the reset kernel
    NA_CK(cudaMemsetAsync(scal, 0, sizeof(NaScalars), s));
    if (ns > 0) {
        NA_CK(cudaMemcpyAsync(dsrc, hsrc, (size_t)ns * sizeof(SourceDev), cudaMemcpyHostToDevice, s));
        NA_CK(launch_make_seeds(dsrc, ns, p->l_base, seeds, s));
    }

    PrepArgs P;
    memset(&P, 0, sizeof P);
    P.n = n;
    P.nb = nb;
    P.ng = G;
    P.nH = nH;
    P.xHI = xHI;
    P.xHeI = xHeI;
    P.xHeII = xHeII;
    P.y = (float)y;
    for (int sp = 0; sp < 3; ++sp)
        for (int b = 0; b < ARC_MAX_GROUPS; ++b)
            P.sig_dx[sp][b] = (b < G) ? (float)(p->sigma[sp][b] * dx) : 0.f;
    P.rec = rec;
    NA_CK(launch_prep(P, s));

    TraceArgs A;
    memset(&A, 0, sizeof A);
    A.n = n;
    A.nb = nb;
    A.bstride_y = (uint32_t)nb << 9;
    A.bstride_x = A.bstride_y * (uint32_t)nb;
    A.ng = G;
    A.l_base = p->l_base;
    A.l_max = p->l_max;
    A.kappa = rec;
    A.acc = rec;
    A.src = dsrc;
    A.nsrc = ns;
    for (int l = 0; l <= ARC_MAX_LEVEL; ++l) A.rsplit[l] = (float)na_r_split(p->phi, l);
    A.seeds = seeds;
    fill_sincos_table(A);
    A.nseeds = nseeds;
    A.seed_head = &scal->seed_head;
    A.qdata = qdata;
    A.qseq = qseq;
    A.qhead = &scal->qhead;
    A.qtail = &scal->qtail;
    A.qmask = NA_QCAP - 1;
    A.live = &scal->live;
    A.n_idle = &scal->n_idle;
    A.status = &scal->status;
    A.heartbeat = &scal->heartbeat;
    A.escaped = &scal->escaped;
    A.rounding = &scal->rounding;
    A.counters = scal->counters;
    A.recs = nullptr;
    A.nrec = &scal->nrec;
    A.rec_cap = 0;
    A.stack_log2 = 8;   // deepest per-warp deques: keeps the small ring from filling
    A.idle_timeout_ns = 10ull * 1000000000ull;
    NA_CK(launch_seed_reset(A, NA_QCAP, nseeds, s));
    if (nseeds > 0) {
        int dev_sms = 0, occ = 0;
        NA_CK(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev));
        const int block = 256;
        const int smem = trace_smem_bytes(block, A.stack_log2);
        NA_CK(cudaFuncSetAttribute(trace_kernel_ptr(G), cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_kernel_ptr(G), block, smem) != cudaSuccess ||
            occ < 1)
            occ = 1;
        NA_CK(launch_trace(A, dev_sms * occ, block, s));
    }

    FinalizeArgs F;
    memset(&F, 0, sizeof F);
    F.n = n;
    F.nb = nb;
    F.ng = G;
    F.nH = nH;
    F.xHI = xHI;
    F.xHeI = xHeI;
    F.xHeII = xHeII;
    F.y = (float)y;
    static const double E_S[3] = {13.6, 24.6, 54.4};
    for (int sp = 0; sp < 3; ++sp)
        for (int b = 0; b < ARC_MAX_GROUPS; ++b) {
            const bool on = b < G;
            F.sig[sp][b] = on ? (float)p->sigma[sp][b] : 0.f;
            F.egap_erg[sp][b] = on ? (float)((p->E_group_eV[b] - E_S[sp]) * EV_ERG) : 0.f;
        }
    F.scale = (float)(PHOT_UNIT / (dx * dx * dx));
    F.rec = rec;
    F.gamma = gamma;
    F.heat = heat;
    F.absorbed_part = parts;
    NA_CK(launch_finalize(F, NA_NPARTS, s));
    NA_CK(launch_budget(parts, NA_NPARTS, &scal->escaped, &scal->rounding, nullptr, scal->budget_out, s));

    // the source table was copied from this stack frame: wait before returning
    NaScalars S;
    NA_CK(cudaMemcpyAsync(&S, scal, sizeof S, cudaMemcpyDeviceToHost, s));
    NA_CK(cudaStreamSynchronize(s));
#undef NA_CK
    if (S.status & (ERR_TIMEOUT | ERR_CAS_SPIN)) return ARC_E_TIMEOUT;
    if (S.status & ERR_QUEUE_FULL) return ARC_E_OVERFLOW;
    double b[4] = {launched, S.budget_out[0] * PHOT_UNIT, S.budget_out[1] * PHOT_UNIT, emitted};
    if (budget)
        for (int i = 0; i < 4; ++i) budget[i] = b[i];
    if (fabs(b[0] - b[1] - b[2]) > 1e-9 * b[0]) return ARC_E_BUDGET;
    return ARC_OK;
}
