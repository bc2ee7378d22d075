// arc_api.cu -- host side of the libarc C ABI (include/arc.h).
//
// Owns the device buffers of a context, validates inputs, orders the kernel
// launches of a step on the context's stream and captures them into a CUDA
// graph for arc_step.  No computation of the method happens here; the FP64
// host arithmetic is limited to parameter set-up (split radii, unit scales)
// and the final budget comparison.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <string>
#include <vector>

#include "arc_internal.cuh"

using namespace arc;

namespace {

struct Scalars {
    unsigned long long qhead, qtail;
    long long live;
    int n_idle;
    unsigned int seed_head;
    unsigned int status;
    unsigned int heartbeat;
    unsigned int pad0;
    double escaped;
    double rounding;
    double thin;                           // photons of the optically thin fill (Sec. 2.6)
    unsigned long long counters[CNT_ALL];
    unsigned long long nrec;
    double budget_out[2];
    unsigned long long chem_counters[4];   // substeps, fp64 substeps, capped, surrogate cells
    unsigned int fb_count;                 // cells sent back to the plain solver
    unsigned int pad1;
};

struct HostSource {
    double pos[3];
    double ndot[ARC_MAX_GROUPS];
    double total;
    uint32_t id;
};

}  // namespace

struct arc_ctx {
    int n = 0, nb = 0;
    double box_cm = 0, dx = 0;
    arc_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;      // created here when the caller passed NULL
    int device = 0, num_sms = 0;
    // fields (C order)
    float *nH = nullptr, *xHI = nullptr, *xHeI = nullptr, *xHeII = nullptr, *T = nullptr;
    // internal brick layout
    float4* rec = nullptr;     // cell records: optical depth, absorbed photons (32 B per cell)
    float *gamma = nullptr, *heat = nullptr;
    // sources
    std::vector<HostSource> hsrc;
    bool src_dirty = true;
    SourceDev* dsrc = nullptr;
    int dsrc_cap = 0, nsrc_dev = 0;
    double launched_rate = 0.0;   // photons/s put into rays (FP64 sum of FP32 shares)
    double emitted_rate = 0.0;    // photons/s of the sources (FP64 input sum)
    Entry* seeds = nullptr;
    int seeds_cap = 0, nseeds = 0;
    std::vector<uint32_t> dev_ids;   // device source order -> caller's index
    // optically thin approximation (Sec. 2.6): radius per device source and
    // the candidates the running trace measures (dsrc_cap entries each)
    float* rthin = nullptr;
    float* rnext = nullptr;
    double last_dt = 0.0;
    // anisotropic escape (Sec. 2.2): caller's mask (caller order) and its copy
    // in device source order
    std::vector<uint8_t> hopen;
    uint8_t* dopen = nullptr;
    size_t dopen_cap = 0;
    // failure-detection test aid (arc_set_fault): unfinished-ray count added at
    // the start of every trace, the value written, and the idle-wait bound
    long long fault_live_bias = 0;
    long long fault_live_value = 0;
    unsigned long long idle_timeout_ns = 10ull * 1000000000ull;
    // dynamic queue
    Entry* qdata = nullptr;
    unsigned long long* qseq = nullptr;
    unsigned long long qcap = 0;
    Scalars* scal = nullptr;
    double* absorbed_part = nullptr;
    int nparts = 152 * 8;
    arc_ray_rec* recs = nullptr;
    long long rec_cap = 0;
    bool fields_set = false, traced = false;
    int block = 256, blocks_per_sm = 0, stack_log2 = 7;
    float rsplit[ARC_MAX_LEVEL + 1] = {};
    cudaGraphExec_t gexec = nullptr;
    double graph_dt = -1.0;
    bool graph_valid = false;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::string err = "no error";
    // chemistry surrogate
    MlpDev* mlp = nullptr;
    bool use_surrogate = false;
    float tol_x = 5e-4f, tol_e = 1e-2f, gate = 0.0f;
    unsigned* fb_list = nullptr;
};

namespace {

arc_status fail(arc_ctx* c, arc_status s, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(c, e_ == cudaErrorMemoryAllocation ? ARC_E_OOM : ARC_E_CUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                       \
    } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
    return cudaMalloc((void**)p, count * sizeof(T));
}

void dfree(void* p) {
    if (p) cudaFree(p);
}

double yfrac(const arc_params& p) { return p.Y / (4.0 * (1.0 - p.Y)); }

arc_status check_params(arc_ctx* c, const arc_grid* g, const arc_params* p) {
    if (!g || !p) return fail(c, ARC_E_INVALID, "null grid or params");
    if (g->n < 1 || g->n > ARC_MAX_N) return fail(c, ARC_E_INVALID, "n=%d outside 1..%d", g->n, ARC_MAX_N);
    if (!(g->box_cm > 0) || !isfinite(g->box_cm)) return fail(c, ARC_E_INVALID, "box_cm must be > 0");
    if (p->ngroups < 1 || p->ngroups > ARC_MAX_GROUPS)
        return fail(c, ARC_E_INVALID, "ngroups=%d outside 1..%d", p->ngroups, ARC_MAX_GROUPS);
    for (int b = 0; b < p->ngroups; ++b) {
        if (!(p->E_group_eV[b] >= 0) || !isfinite(p->E_group_eV[b]))
            return fail(c, ARC_E_INVALID, "E_group_eV[%d] invalid", b);
        for (int s = 0; s < 3; ++s)
            if (!(p->sigma[s][b] >= 0) || !isfinite(p->sigma[s][b]))
                return fail(c, ARC_E_INVALID, "sigma[%d][%d] invalid", s, b);
    }
    if (!(p->Y >= 0 && p->Y < 1)) return fail(c, ARC_E_INVALID, "Y outside [0,1)");
    if (!(p->phi > 0) || !isfinite(p->phi)) return fail(c, ARC_E_INVALID, "phi must be > 0");
    if (p->l_base < 1 || p->l_base > 6) return fail(c, ARC_E_INVALID, "l_base outside 1..6");
    if (p->geo_correction != 0 && p->geo_correction != 1)
        return fail(c, ARC_E_INVALID, "geo_correction must be 0 or 1");
    if (p->thin_approx != 0 && p->thin_approx != 1) return fail(c, ARC_E_INVALID, "thin_approx must be 0 or 1");
    if (p->thin_approx)
        for (int b = 1; b < p->ngroups; ++b)
            if (p->E_group_eV[b] < p->E_group_eV[0])
                return fail(c, ARC_E_INVALID, "thin_approx needs group 0 to be the softest");
    if (p->l_max < p->l_base || p->l_max > ARC_MAX_LEVEL)
        return fail(c, ARC_E_INVALID, "l_max outside l_base..%d", ARC_MAX_LEVEL);
    if (!(p->term_frac > 0 && p->term_frac < 1)) return fail(c, ARC_E_INVALID, "term_frac outside (0,1)");
    if (!(p->eps_sub > 0 && p->eps_sub <= 1)) return fail(c, ARC_E_INVALID, "eps_sub outside (0,1]");
    if (!(p->x_fp64 > 0 && p->x_fp64 < 1)) return fail(c, ARC_E_INVALID, "x_fp64 outside (0,1)");
    if (!(p->alpha_B_fixed >= 0)) return fail(c, ARC_E_INVALID, "alpha_B_fixed < 0");
    return ARC_OK;
}

// split distance (Sec. 2.4): a level-l ray covers 4 pi / (12 4^l) sr; fewer than
// phi rays cross a unit cell face beyond r = 1 / sqrt(phi Omega_l).
double r_split(double phi, int level) {
    const double omega = 4.0 * M_PI / (12.0 * pow(4.0, level));
    return 1.0 / sqrt(phi * omega);
}

arc_status sync_status(arc_ctx* c, Scalars* out) {
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaMemcpy(out, c->scal, sizeof(Scalars), cudaMemcpyDeviceToHost));
    return ARC_OK;
}

arc_status status_to_error(arc_ctx* c, unsigned st) {
    if (st & ERR_TIMEOUT) return fail(c, ARC_E_TIMEOUT, "tracer: an idle warp gave up waiting (status 0x%x)", st);
    if (st & ERR_CAS_SPIN) return fail(c, ARC_E_TIMEOUT, "tracer: queue CAS loop bound hit (status 0x%x)", st);
    if (st & ERR_QUEUE_FULL) return fail(c, ARC_E_OVERFLOW, "tracer: global work queue full (status 0x%x)", st);
    if (st & ERR_RECORDS) return fail(c, ARC_E_OVERFLOW, "tracer: ray record buffer full (status 0x%x)", st);
    if (st & ERR_SUBSTEP) return fail(c, ARC_E_SUBSTEP, "chemistry: a cell hit the sub-step cap (status 0x%x)", st);
    return ARC_OK;
}

// upload the source table (sorted brightest first) and the emitted work items
arc_status upload_sources(arc_ctx* c) {
    if (!c->src_dirty) return ARC_OK;
    std::vector<const HostSource*> act;
    for (const auto& s : c->hsrc)
        if (s.total > 0) act.push_back(&s);
    std::stable_sort(act.begin(), act.end(),
                     [](const HostSource* a, const HostSource* b) { return a->total > b->total; });
    const int G = c->p.ngroups;
    const double nrays = 12.0 * pow(4.0, c->p.l_base);
    const int nbase = 12 << (2 * c->p.l_base);
    const bool masked = !c->hopen.empty();
    std::vector<SourceDev> h(act.size());
    std::vector<uint8_t> dmask(masked ? act.size() * (size_t)nbase : 0);
    c->dev_ids.resize(act.size());
    double launched = 0.0, emitted = 0.0;
    for (size_t i = 0; i < act.size(); ++i) {
        const HostSource& s = *act[i];
        int open = nbase;
        if (masked) {
            open = 0;
            for (int q = 0; q < nbase; ++q) {
                const uint8_t v = c->hopen[(size_t)s.id * nbase + q] ? 1 : 0;
                dmask[i * (size_t)nbase + q] = v;
                open += v;
            }
        }
        float N0[ARC_MAX_GROUPS] = {0.f, 0.f, 0.f, 0.f};
        double tot = 0.0;
        for (int b = 0; b < G; ++b) {
            N0[b] = (float)(s.ndot[b] / PHOT_UNIT / nrays);
            launched += (double)N0[b] * open * PHOT_UNIT;   // blocked rays carry nothing
            tot += (double)N0[b];
        }
        emitted += s.total;
        float ph[3], pl[3];
        for (int a = 0; a < 3; ++a) {   // the FP64 position as an FP32 pair
            ph[a] = (float)s.pos[a];
            pl[a] = (float)(s.pos[a] - (double)ph[a]);
        }
        h[i].pos_thr = make_float4(ph[0], ph[1], ph[2], (float)(c->p.term_frac * tot));
        h[i].N0 = make_float4(N0[0], N0[1], N0[2], N0[3]);
        h[i].pos_lo = make_float4(pl[0], pl[1], pl[2],
                                  N0[0] > 0.f ? (float)((double)N0[0] * exp(-0.1)) : 0.f);   // Sec. 2.6
        h[i].id = s.id;
        h[i].pad[0] = h[i].pad[1] = h[i].pad[2] = 0;
        c->dev_ids[i] = s.id;
    }
    const int ns = (int)act.size();
    const int per_src = 3 << (2 * c->p.l_base);
    if (ns > c->dsrc_cap) {
        dfree(c->dsrc);
        dfree(c->rthin);
        dfree(c->rnext);
        c->dsrc = nullptr;
        c->rthin = c->rnext = nullptr;
        const int cap = std::max(ns, 16);
        CK(dalloc(&c->dsrc, cap));
        CK(dalloc(&c->rthin, cap));
        CK(dalloc(&c->rnext, cap));
        c->dsrc_cap = cap;
        c->graph_valid = false;
    }
    if (masked && dmask.size() > c->dopen_cap) {
        dfree(c->dopen);
        c->dopen = nullptr;
        CK(dalloc(&c->dopen, dmask.size()));
        c->dopen_cap = dmask.size();
        c->graph_valid = false;
    }
    if ((long long)ns * per_src > c->seeds_cap) {
        dfree(c->seeds);
        c->seeds = nullptr;
        const long long cap = std::max<long long>((long long)ns * per_src, 64);
        if (cap > (1ll << 30)) return fail(c, ARC_E_INVALID, "too many sources");
        CK(dalloc(&c->seeds, (size_t)cap));
        c->seeds_cap = (int)cap;
        c->graph_valid = false;
    }
    if (ns > 0) {
        CK(cudaMemcpyAsync(c->dsrc, h.data(), ns * sizeof(SourceDev), cudaMemcpyHostToDevice, c->stream));
        if (masked)
            CK(cudaMemcpyAsync(c->dopen, dmask.data(), dmask.size(), cudaMemcpyHostToDevice, c->stream));
        // a new source table starts every optically thin radius at 0
        CK(cudaMemsetAsync(c->rthin, 0, ns * sizeof(float), c->stream));
        CK(launch_make_seeds(c->dsrc, ns, c->p.l_base, c->seeds, c->stream));
        CK(cudaStreamSynchronize(c->stream));   // h and dmask go out of scope
    }
    if (ns != c->nsrc_dev) c->graph_valid = false;
    c->nsrc_dev = ns;
    c->nseeds = ns * per_src;
    c->launched_rate = launched;
    c->emitted_rate = emitted;
    c->src_dirty = false;
    return ARC_OK;
}

// Events inside a captured graph must be external record nodes; outside a
// capture they are plain records.
cudaError_t record_event(arc_ctx* c, cudaEvent_t ev) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(c->stream, &cs);
    if (e != cudaSuccess) return e;
    if (cs == cudaStreamCaptureStatusActive)
        return cudaEventRecordWithFlags(ev, c->stream, cudaEventRecordExternal);
    return cudaEventRecord(ev, c->stream);
}

TraceArgs trace_args(arc_ctx* c) {
    TraceArgs a;
    memset(&a, 0, sizeof a);
    a.n = c->n;
    a.nb = c->nb;
    a.bstride_y = (uint32_t)c->nb << 9;
    a.bstride_x = a.bstride_y * (uint32_t)c->nb;
    a.ng = c->p.ngroups;
    a.l_base = c->p.l_base;
    a.l_max = c->p.l_max;
    a.kappa = c->rec;
    a.acc = c->rec;
    a.src = c->dsrc;
    a.nsrc = c->nsrc_dev;
    for (int l = 0; l <= ARC_MAX_LEVEL; ++l) {
        a.rsplit[l] = c->rsplit[l];
        a.pixw[l] = (float)sqrt(4.0 * M_PI / (12.0 * ldexp(1.0, 2 * l)));   // Omega_l = 4 pi / (12 4^l)
    }
    a.geo_corr = c->p.geo_correction ? 1 : 0;
    fill_sincos_table(a);
    a.open = c->hopen.empty() ? nullptr : c->dopen;
    a.nbase = 12 << (2 * c->p.l_base);
    a.rnext = c->p.thin_approx ? c->rnext : nullptr;
    a.thin = &c->scal->thin;
    a.seeds = c->seeds;
    a.nseeds = c->nseeds;
    a.seed_head = &c->scal->seed_head;
    a.qdata = c->qdata;
    a.qseq = c->qseq;
    a.qhead = &c->scal->qhead;
    a.qtail = &c->scal->qtail;
    a.qmask = c->qcap - 1;
    a.live = &c->scal->live;
    a.n_idle = &c->scal->n_idle;
    a.status = &c->scal->status;
    a.heartbeat = &c->scal->heartbeat;
    a.escaped = &c->scal->escaped;
    a.rounding = &c->scal->rounding;
    a.counters = c->scal->counters;
    a.recs = c->recs;
    a.nrec = &c->scal->nrec;
    a.rec_cap = (unsigned long long)c->rec_cap;
    a.stack_log2 = c->stack_log2;
    a.idle_timeout_ns = c->idle_timeout_ns;
    return a;
}

int trace_grid(arc_ctx* c) {
    int per_sm = c->blocks_per_sm;
    if (per_sm <= 0) {
        int occ = 0;
        const int smem = trace_smem_bytes(c->block, c->stack_log2);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_kernel_ptr(c->p.ngroups, false,
                                                                           c->p.thin_approx || !c->hopen.empty()),
                                                          c->block, smem) !=
                cudaSuccess ||
            occ < 1)
            occ = 1;
        per_sm = occ;
    }
    return c->num_sms * per_sm;
}

// queue the trace of the current fields on the context stream (no sync);
// seeds_limit > 0 traces only the first seeds_limit emitted items (the
// brightest sources), used by the autotuner
arc_status enqueue_trace(arc_ctx* c, int seeds_limit = 0) {
    PrepArgs P;
    memset(&P, 0, sizeof P);
    P.n = c->n;
    P.nb = c->nb;
    P.ng = c->p.ngroups;
    P.nH = c->nH;
    P.xHI = c->xHI;
    P.xHeI = c->xHeI;
    P.xHeII = c->xHeII;
    P.y = (float)yfrac(c->p);
    for (int s = 0; s < 3; ++s)
        for (int b = 0; b < ARC_MAX_GROUPS; ++b)
            P.sig_dx[s][b] = (b < c->p.ngroups) ? (float)(c->p.sigma[s][b] * c->dx) : 0.f;
    P.rec = c->rec;
    CK(launch_prep(P, c->stream));
    TraceArgs A = trace_args(c);
    if (seeds_limit > 0 && seeds_limit < A.nseeds) A.nseeds = seeds_limit;
    CK(launch_seed_reset(A, c->qcap, A.nseeds, c->stream));
    if (c->fault_live_bias != 0) {
        // test aid: a count of unfinished rays that can never reach zero, so
        // that idle warps wait for work that never comes (arc_set_fault)
        c->fault_live_value = 4ll * A.nseeds + c->fault_live_bias;
        CK(cudaMemcpyAsync(&c->scal->live, &c->fault_live_value, sizeof(long long), cudaMemcpyHostToDevice,
                           c->stream));
    }
    CK(record_event(c, c->ev[0]));
    if (c->p.thin_approx && c->nsrc_dev > 0) {
        // Sec. 2.6: rays start at each source's radius; the cells inside it
        // take the thin-limit absorption
        CK(launch_thin_begin(c->seeds, A.nseeds, c->rthin, c->rnext, c->nsrc_dev, c->stream));
        ThinFillArgs T;
        T.n = c->n;
        T.nb = c->nb;
        T.nsrc = c->nsrc_dev;
        T.src = c->dsrc;
        T.rthin = c->rthin;
        T.nbase = (float)(12 << (2 * c->p.l_base));
        T.rec = c->rec;
        T.thin = &c->scal->thin;
        T.rounding = &c->scal->rounding;
        CK(launch_thin_fill(T, c->stream));
    }
    if (A.nseeds > 0) CK(launch_trace(A, trace_grid(c), c->block, c->stream));
    // the autotuner's partial traces (seeds_limit) leave the radii as they are
    if (c->p.thin_approx && c->nsrc_dev > 0 && seeds_limit == 0)
        CK(launch_thin_commit(c->rthin, c->rnext, c->nsrc_dev, c->stream));
    CK(record_event(c, c->ev[1]));
    FinalizeArgs F;
    memset(&F, 0, sizeof F);
    F.n = c->n;
    F.nb = c->nb;
    F.ng = c->p.ngroups;
    F.nH = c->nH;
    F.xHI = c->xHI;
    F.xHeI = c->xHeI;
    F.xHeII = c->xHeII;
    F.y = (float)yfrac(c->p);
    static const double E_S[3] = {13.6, 24.6, 54.4};
    for (int s = 0; s < 3; ++s)
        for (int b = 0; b < ARC_MAX_GROUPS; ++b) {
            const bool on = b < c->p.ngroups;
            F.sig[s][b] = on ? (float)c->p.sigma[s][b] : 0.f;
            F.egap_erg[s][b] = on ? (float)((c->p.E_group_eV[b] - E_S[s]) * EV_ERG) : 0.f;
        }
    F.scale = (float)(PHOT_UNIT / (c->dx * c->dx * c->dx));
    F.rec = c->rec;
    F.gamma = c->gamma;
    F.heat = c->heat;
    F.absorbed_part = c->absorbed_part;
    CK(launch_finalize(F, c->nparts, c->stream));
    CK(launch_budget(c->absorbed_part, c->nparts, &c->scal->escaped, &c->scal->rounding, &c->scal->thin,
                     c->scal->budget_out, c->stream));
    return ARC_OK;
}

// chemistry switches and coefficients of the context (state arrays left to the caller)
ChemArgs chem_args(const arc_ctx* c, double dt) {
    ChemArgs C;
    memset(&C, 0, sizeof C);
    C.dt = dt;
    C.y = (float)yfrac(c->p);
    C.eps = (float)c->p.eps_sub;
    C.xfloor = (float)c->p.x_fp64;
    C.alpha_fixed = (float)c->p.alpha_B_fixed;
    C.isothermal = c->p.isothermal;
    C.coll_ion = c->p.coll_ion;
    C.compton = c->p.z_compton >= 0 ? 1 : 0;
    const double tg = 2.725 * (1.0 + (c->p.z_compton >= 0 ? c->p.z_compton : 0.0));
    C.tcmb = (float)tg;
    // 4 sigma_T a k / (m_e c) T_g^4 [erg/s/K per electron]
    C.compton_coef = (float)(4.0 * 6.6524587e-25 * 7.5657e-15 * K_BOLTZ / (9.1093837e-28 * 2.99792458e10) *
                             tg * tg * tg * tg);
    return C;
}

arc_status enqueue_chem(arc_ctx* c, double dt) {
    ChemArgs C = chem_args(c, dt);
    C.ncell = (long long)c->n * c->n * c->n;
    C.nH = c->nH;
    C.xHI = c->xHI;
    C.xHeI = c->xHeI;
    C.xHeII = c->xHeII;
    C.T = c->T;
    C.gamma = c->gamma;
    C.heat = c->heat;
    C.status = &c->scal->status;
    C.counters = c->scal->chem_counters;
    C.list = nullptr;
    C.list_count = nullptr;
    CK(cudaMemsetAsync(c->scal->chem_counters, 0, sizeof(c->scal->chem_counters), c->stream));
    CK(cudaMemsetAsync(&c->scal->fb_count, 0, sizeof(unsigned), c->stream));
    CK(record_event(c, c->ev[2]));
    if (c->use_surrogate) {
        // network step for every cell; rejected cells -> plain sub-cycled solver
        SurrogateArgs S;
        S.w = c->mlp;
        S.tol_x = c->tol_x;
        S.tol_e = c->tol_e;
        S.gate = c->gate;
        S.fb_list = c->fb_list;
        S.fb_count = &c->scal->fb_count;
        CK(launch_chem_surrogate(C, S, c->stream));
        C.list = c->fb_list;
        C.list_count = &c->scal->fb_count;
    }
    CK(launch_chem(C, c->stream));
    CK(record_event(c, c->ev[3]));
    return ARC_OK;
}

}  // namespace

extern "C" {

arc_status arc_create(arc_ctx** out, const arc_grid* g, const arc_params* p, void* stream) {
    if (!out) return ARC_E_INVALID;
    *out = nullptr;
    arc_ctx* c = new arc_ctx();
    arc_status st = check_params(c, g, p);
    if (st != ARC_OK) {
        delete c;
        return st;
    }
    c->n = g->n;
    c->nb = (g->n + 7) / 8;
    c->box_cm = g->box_cm;
    c->dx = g->box_cm / g->n;
    c->p = *p;
    c->stream = (cudaStream_t)stream;
    for (int l = 0; l <= ARC_MAX_LEVEL; ++l) c->rsplit[l] = (float)r_split(p->phi, l);
    auto bail = [&](arc_status s) {
        arc_destroy(c);
        return s;
    };
    if (!c->stream) {
        // a private stream: the legacy default stream cannot be captured into a graph
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(ARC_E_CUDA);
        c->own_stream = true;
    }
    // allow the largest tuning (256 threads x 256 deque entries) once, for every context
    for (int ng : {1, 3, 4})
        for (bool rec : {false, true})
            for (bool ext : {false, true})
                if (cudaFuncSetAttribute(trace_kernel_ptr(ng, rec, ext), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         trace_smem_bytes(256, 8)) != cudaSuccess)
                    return bail(ARC_E_CUDA);
    if (cudaGetDevice(&c->device) != cudaSuccess) return bail(ARC_E_CUDA);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(ARC_E_CUDA);
    const size_t n3 = (size_t)c->n * c->n * c->n;
    const size_t nbc = (size_t)c->nb * c->nb * c->nb * 512;
    cudaError_t e = cudaSuccess;
    e = e ? e : dalloc(&c->nH, n3);
    e = e ? e : dalloc(&c->xHI, n3);
    e = e ? e : dalloc(&c->xHeI, n3);
    e = e ? e : dalloc(&c->xHeII, n3);
    e = e ? e : dalloc(&c->T, n3);
    e = e ? e : dalloc(&c->rec, 2 * nbc);
    e = e ? e : dalloc(&c->gamma, 3 * n3);
    e = e ? e : dalloc(&c->heat, 3 * n3);
    c->qcap = 1ull << 22;
    e = e ? e : dalloc(&c->qdata, c->qcap);
    e = e ? e : dalloc(&c->qseq, c->qcap);
    e = e ? e : dalloc(&c->scal, 1);
    e = e ? e : dalloc(&c->absorbed_part, c->nparts);
    if (e != cudaSuccess) return bail(e == cudaErrorMemoryAllocation ? ARC_E_OOM : ARC_E_CUDA);
    e = cudaMemsetAsync(c->scal, 0, sizeof(Scalars), c->stream);
    e = e ? e : cudaMemsetAsync(c->gamma, 0, 3 * n3 * sizeof(float), c->stream);
    e = e ? e : cudaMemsetAsync(c->heat, 0, 3 * n3 * sizeof(float), c->stream);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
    e = e ? e : cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(ARC_E_CUDA);
    *out = c;
    return ARC_OK;
}

arc_status arc_set_fields(arc_ctx* c, const float* nH, const float* xHI, const float* xHeI,
                          const float* xHeII, const float* T, int on_device) {
    if (!c) return ARC_E_INVALID;
    if (!nH || !xHI || !xHeI || !xHeII || !T) return fail(c, ARC_E_INVALID, "null field pointer");
    const size_t n3 = (size_t)c->n * c->n * c->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const float* src[5] = {nH, xHI, xHeI, xHeII, T};
    float* dst[5] = {c->nH, c->xHI, c->xHeI, c->xHeII, c->T};
    for (int i = 0; i < 5; ++i) CK(cudaMemcpyAsync(dst[i], src[i], n3 * sizeof(float), kind, c->stream));
    CK(cudaMemsetAsync(&c->scal->status, 0, sizeof(unsigned), c->stream));
    CK(launch_validate(c->nH, c->xHI, c->xHeI, c->xHeII, c->T, (long long)n3, &c->scal->status, c->stream));
    unsigned st = 0;
    CK(cudaMemcpyAsync(&st, &c->scal->status, sizeof st, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (st & ERR_FIELDS) {
        c->fields_set = false;
        return fail(c, ARC_E_INVALID,
                    "field values out of range (need finite, nH>=0, fractions in [0,1], xHeI+xHeII<=1, T>0)");
    }
    c->fields_set = true;
    return ARC_OK;
}

arc_status arc_add_sources(arc_ctx* c, int nsrc, const double* pos, const double* ndot) {
    if (!c) return ARC_E_INVALID;
    if (nsrc < 0 || (nsrc > 0 && (!pos || !ndot))) return fail(c, ARC_E_INVALID, "bad source arrays");
    const int G = c->p.ngroups;
    for (int i = 0; i < nsrc; ++i) {
        HostSource s;
        memset(&s, 0, sizeof s);
        for (int a = 0; a < 3; ++a) {
            s.pos[a] = pos[3 * i + a];
            if (!(s.pos[a] >= 0.0 && s.pos[a] < (double)c->n))
                return fail(c, ARC_E_INVALID, "source %d position outside the box", i);
        }
        for (int b = 0; b < G; ++b) {
            s.ndot[b] = ndot[(size_t)i * G + b];
            if (!(s.ndot[b] >= 0.0) || !isfinite(s.ndot[b]))
                return fail(c, ARC_E_INVALID, "source %d rate invalid", i);
            s.total += s.ndot[b];
        }
        s.id = (uint32_t)c->hsrc.size();
        c->hsrc.push_back(s);
    }
    c->hopen.clear();   // a mask covers the sources it was set for
    c->src_dirty = true;
    c->graph_valid = false;
    return ARC_OK;
}

arc_status arc_clear_sources(arc_ctx* c) {
    if (!c) return ARC_E_INVALID;
    c->hsrc.clear();
    c->hopen.clear();
    c->src_dirty = true;
    c->graph_valid = false;
    return ARC_OK;
}

arc_status arc_trace(arc_ctx* c, double dt, float** gamma, float** heat, double* budget) {
    if (!c) return ARC_E_INVALID;
    if (!c->fields_set) return fail(c, ARC_E_STATE, "arc_set_fields must come first");
    if (!(dt >= 0) || !isfinite(dt)) return fail(c, ARC_E_INVALID, "dt invalid");
    arc_status st = upload_sources(c);
    if (st != ARC_OK) return st;
    st = enqueue_trace(c);
    if (st != ARC_OK) return st;
    c->traced = true;
    c->last_dt = dt;
    if (gamma) *gamma = c->gamma;
    if (heat) *heat = c->heat;
    if (budget) {
        Scalars S;
        st = sync_status(c, &S);
        if (st != ARC_OK) return st;
        budget[0] = c->launched_rate * dt;
        budget[1] = S.budget_out[0] * PHOT_UNIT * dt;
        budget[2] = S.budget_out[1] * PHOT_UNIT * dt;
        budget[3] = c->emitted_rate * dt;
        st = status_to_error(c, S.status);
        if (st != ARC_OK) return st;
        const double resid = fabs(budget[0] - budget[1] - budget[2]);
        if (resid > 1e-9 * budget[0])
            return fail(c, ARC_E_BUDGET, "photon budget off by %.3e of the launched photons",
                        budget[0] > 0 ? resid / budget[0] : resid);
    }
    return ARC_OK;
}

arc_status arc_chem_update(arc_ctx* c, double dt) {
    if (!c) return ARC_E_INVALID;
    if (!c->fields_set) return fail(c, ARC_E_STATE, "arc_set_fields must come first");
    if (!(dt >= 0) || !isfinite(dt)) return fail(c, ARC_E_INVALID, "dt invalid");
    return enqueue_chem(c, dt);
}

arc_status arc_step(arc_ctx* c, double dt) {
    if (!c) return ARC_E_INVALID;
    if (!c->fields_set) return fail(c, ARC_E_STATE, "arc_set_fields must come first");
    if (!(dt >= 0) || !isfinite(dt)) return fail(c, ARC_E_INVALID, "dt invalid");
    arc_status st = upload_sources(c);
    if (st != ARC_OK) return st;
    if (!c->graph_valid || c->graph_dt != dt) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        cudaGraph_t g = nullptr;
        CK(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
        arc_status s1 = enqueue_trace(c);
        arc_status s2 = (s1 == ARC_OK) ? enqueue_chem(c, dt) : s1;
        cudaError_t ee = cudaStreamEndCapture(c->stream, &g);
        if (s2 != ARC_OK) {
            if (g) cudaGraphDestroy(g);
            return s2;
        }
        if (ee != cudaSuccess) return fail(c, ARC_E_CUDA, "graph capture: %s", cudaGetErrorString(ee));
        ee = cudaGraphInstantiate(&c->gexec, g, 0);
        cudaGraphDestroy(g);
        if (ee != cudaSuccess) return fail(c, ARC_E_CUDA, "graph instantiate: %s", cudaGetErrorString(ee));
        c->graph_valid = true;
        c->graph_dt = dt;
    }
    CK(cudaGraphLaunch(c->gexec, c->stream));
    c->traced = true;
    return ARC_OK;
}

arc_status arc_get_fields(arc_ctx* c, float* xHI, float* xHeI, float* xHeII, float* T, int on_device) {
    if (!c) return ARC_E_INVALID;
    const size_t n3 = (size_t)c->n * c->n * c->n;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    float* dst[4] = {xHI, xHeI, xHeII, T};
    const float* src[4] = {c->xHI, c->xHeI, c->xHeII, c->T};
    for (int i = 0; i < 4; ++i)
        if (dst[i]) CK(cudaMemcpyAsync(dst[i], src[i], n3 * sizeof(float), kind, c->stream));
    Scalars S;
    arc_status st = sync_status(c, &S);
    if (st != ARC_OK) return st;
    return status_to_error(c, S.status);
}

arc_status arc_set_records(arc_ctx* c, void* buf, int64_t cap) {
    if (!c) return ARC_E_INVALID;
    if (cap < 0 || (buf && cap == 0)) return fail(c, ARC_E_INVALID, "bad record capacity");
    c->recs = (arc_ray_rec*)buf;
    c->rec_cap = buf ? cap : 0;
    c->graph_valid = false;
    return ARC_OK;
}

arc_status arc_get_record_count(arc_ctx* c, int64_t* count) {
    if (!c || !count) return ARC_E_INVALID;
    Scalars S;
    arc_status st = sync_status(c, &S);
    if (st != ARC_OK) return st;
    *count = (int64_t)S.nrec;
    return ARC_OK;
}

arc_status arc_stats(arc_ctx* c, arc_stats_t* out) {
    if (!c || !out) return ARC_E_INVALID;
    Scalars S;
    arc_status st = sync_status(c, &S);
    if (st != ARC_OK) return st;
    memset(out, 0, sizeof *out);
    out->segments = S.counters[CNT_SEG];
    out->rays = S.counters[CNT_RAYS];
    out->splits = S.counters[CNT_SPLIT];
    out->terminated = S.counters[CNT_TERM];
    out->escaped_rays = S.counters[CNT_ESC];
    out->donations = S.counters[CNT_DONATE];
    out->max_level = (uint32_t)S.counters[CNT_MAXLEVEL];
    out->error_word = S.status;
    out->chem_substeps = S.chem_counters[0];
    out->chem_fp64_substeps = S.chem_counters[1];
    out->chem_capped = S.chem_counters[2];
    out->segments_total = S.counters[CNT_SEG_TOTAL];
    out->traces_total = S.counters[CNT_TRACES_TOTAL];
    out->surrogate_cells = S.chem_counters[3];
    out->fallback_cells = c->use_surrogate ? S.fb_count : 0;
    float ms = 0.f;
    if (c->traced && cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]) == cudaSuccess) out->trace_ms = ms;
    if (cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]) == cudaSuccess) out->chem_ms = ms;
    cudaGetLastError();   // elapsed-time queries on unrecorded events are not errors here
    return ARC_OK;
}

arc_status arc_get_tuning(arc_ctx* c, int* block_threads, int* blocks_per_sm, int* stack_entries) {
    if (!c) return ARC_E_INVALID;
    if (block_threads) *block_threads = c->block;
    if (blocks_per_sm) *blocks_per_sm = c->blocks_per_sm > 0 ? c->blocks_per_sm : trace_grid(c) / c->num_sms;
    if (stack_entries) *stack_entries = 1 << c->stack_log2;
    return ARC_OK;
}

arc_status arc_set_tuning(arc_ctx* c, int block_threads, int blocks_per_sm, int stack_entries) {
    if (!c) return ARC_E_INVALID;
    if (block_threads) {
        if (block_threads < 64 || block_threads > 256 || block_threads % 32)
            return fail(c, ARC_E_INVALID, "block_threads must be a multiple of 32 in 64..256");
        c->block = block_threads;
    }
    if (blocks_per_sm < 0 || blocks_per_sm > 32) return fail(c, ARC_E_INVALID, "blocks_per_sm outside 0..32");
    c->blocks_per_sm = blocks_per_sm;
    if (stack_entries) {
        int lg = 0;
        while ((1 << lg) < stack_entries) ++lg;
        if ((1 << lg) != stack_entries || lg < 6 || lg > 8)
            return fail(c, ARC_E_INVALID, "stack_entries must be a power of two in 64..256");
        c->stack_log2 = lg;
    }
    c->graph_valid = false;
    return ARC_OK;
}

arc_status arc_set_surrogate(arc_ctx* c, const float* params, const float* norm, double tol_x, double tol_e,
                             double gate) {
    if (!c) return ARC_E_INVALID;
    if (!params) {
        c->use_surrogate = false;
        c->graph_valid = false;
        return ARC_OK;
    }
    if (!norm || !(tol_x > 0) || !(tol_e > 0) || !(gate >= 0) || !isfinite(gate))
        return fail(c, ARC_E_INVALID, "surrogate: bad norm, tolerances or gate");
    for (int i = 0; i < ARC_MLP_NNORM; ++i)
        if (!isfinite(norm[i]) || (((i >= MLP_IN && i < 2 * MLP_IN) || i >= 2 * MLP_IN + MLP_OUT) && !(norm[i] > 0)))
            return fail(c, ARC_E_INVALID, "surrogate: normalisation entry %d invalid", i);
    const size_t n3 = (size_t)c->n * c->n * c->n;
    if (!c->mlp) CK(dalloc(&c->mlp, 1));
    if (!c->fb_list) CK(dalloc(&c->fb_list, n3));
    float* dp = nullptr;
    CK(dalloc(&dp, (size_t)MLP_NPARAMS + ARC_MLP_NNORM));
    cudaError_t e = cudaMemcpyAsync(dp, params, MLP_NPARAMS * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dp + MLP_NPARAMS, norm, ARC_MLP_NNORM * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = launch_pack_mlp(dp, dp + MLP_NPARAMS, c->mlp, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(dp);
    if (e != cudaSuccess) return fail(c, ARC_E_CUDA, "surrogate upload: %s", cudaGetErrorString(e));
    c->tol_x = (float)tol_x;
    c->tol_e = (float)tol_e;
    c->gate = (float)gate;
    c->use_surrogate = true;
    c->graph_valid = false;
    return ARC_OK;
}

arc_status arc_rt_timestep(arc_ctx* c, double eps, double* dt_n, double* dt_I) {
    if (!c) return ARC_E_INVALID;
    if (!c->fields_set) return fail(c, ARC_E_STATE, "arc_set_fields must come first");
    if (!(eps > 0) || !isfinite(eps) || !dt_n || !dt_I) return fail(c, ARC_E_INVALID, "eps <= 0 or null output");
    ChemArgs C = chem_args(c, 0.0);
    C.ncell = (long long)c->n * c->n * c->n;
    C.nH = c->nH;
    C.xHI = c->xHI;
    C.xHeI = c->xHeI;
    C.xHeII = c->xHeII;
    C.T = c->T;
    C.gamma = c->gamma;   // Gamma_HI of the last trace (zero before any trace)
    unsigned* out = nullptr;
    CK(dalloc(&out, 2));
    const unsigned inf_bits[2] = {0x7f800000u, 0x7f800000u};
    cudaError_t e = cudaMemcpyAsync(out, inf_bits, sizeof inf_bits, cudaMemcpyHostToDevice, c->stream);
    const float sigd = (float)(c->p.sigma[0][0] * c->dx);
    if (e == cudaSuccess) e = launch_rt_timestep(C, sigd, (float)eps, out, c->stream);
    unsigned bits[2] = {0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits, out, sizeof bits, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(out);
    if (e != cudaSuccess) return fail(c, ARC_E_CUDA, "arc_rt_timestep: %s", cudaGetErrorString(e));
    float f[2];
    memcpy(f, bits, sizeof f);
    *dt_n = (double)f[0];
    *dt_I = (double)f[1];
    return ARC_OK;
}

arc_status arc_mlp_targets(arc_ctx* c, const float* nH, const float* x0, const float* T0, const float* gamma,
                           const float* heat, const float* x1, const float* T1, double dt, long long n, float* Y) {
    if (!c) return ARC_E_INVALID;
    if (!nH || !x0 || !T0 || !gamma || !heat || !x1 || !T1 || !Y || n < 1 || !(dt > 0) || !isfinite(dt))
        return fail(c, ARC_E_INVALID, "arc_mlp_targets: null array, n < 1 or bad dt");
    ChemArgs C = chem_args(c, dt);
    C.ncell = n;
    C.nH = const_cast<float*>(nH);
    C.xHI = const_cast<float*>(x0);
    C.xHeI = const_cast<float*>(x0 + n);
    C.xHeII = const_cast<float*>(x0 + 2 * n);
    C.T = const_cast<float*>(T0);
    C.gamma = gamma;
    C.heat = heat;
    cudaError_t e = launch_mlp_targets(C, x1, T1, Y, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, ARC_E_CUDA, "arc_mlp_targets: %s", cudaGetErrorString(e));
    return ARC_OK;
}

arc_status arc_autotune(arc_ctx* c, int max_sources, int reps, double* best_ms) {
    if (!c) return ARC_E_INVALID;
    if (!c->fields_set) return fail(c, ARC_E_STATE, "arc_set_fields must come first");
    if (reps < 1 || reps > 16) return fail(c, ARC_E_INVALID, "reps outside 1..16");
    arc_status st = upload_sources(c);
    if (st != ARC_OK) return st;
    const int per_src = 3 << (2 * c->p.l_base);
    const int limit = (max_sources > 0) ? max_sources * per_src : 0;
    const int blocks[2] = {128, 256};
    const int stacks[3] = {6, 7, 8};
    const int save_block = c->block, save_bps = c->blocks_per_sm, save_stack = c->stack_log2;
    double best = 1e300;
    int bb = save_block, bbps = save_bps, bst = save_stack;
    for (int bi = 0; bi < 2; ++bi)
        for (int si = 0; si < 3; ++si) {
            int occ = 0;
            const int smem = trace_smem_bytes(blocks[bi], stacks[si]);
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, trace_kernel_ptr(c->p.ngroups), blocks[bi],
                                                              smem) != cudaSuccess || occ < 1)
                continue;
            for (int bps = occ; bps >= 1 && bps >= occ - 1; --bps) {
                c->block = blocks[bi];
                c->blocks_per_sm = bps;
                c->stack_log2 = stacks[si];
                double tot = 0.0;
                for (int r = 0; r < reps; ++r) {
                    st = enqueue_trace(c, limit);
                    if (st != ARC_OK) break;
                    CK(cudaStreamSynchronize(c->stream));
                    float ms = 0.f;
                    CK(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
                    tot += ms;
                }
                if (st != ARC_OK) break;
                Scalars S;
                st = sync_status(c, &S);
                if (st == ARC_OK) st = status_to_error(c, S.status);
                if (st != ARC_OK) break;
                if (tot / reps < best) {
                    best = tot / reps;
                    bb = c->block;
                    bbps = bps;
                    bst = c->stack_log2;
                }
            }
            if (st != ARC_OK) break;
        }
    if (st != ARC_OK) {
        c->block = save_block;
        c->blocks_per_sm = save_bps;
        c->stack_log2 = save_stack;
        return st;
    }
    c->block = bb;
    c->blocks_per_sm = bbps;
    c->stack_log2 = bst;
    c->graph_valid = false;
    if (best_ms) *best_ms = best;
    return ARC_OK;
}

const char* arc_last_error(const arc_ctx* c) { return c ? c->err.c_str() : "null context"; }

arc_status arc_set_emission_mask(arc_ctx* c, const uint8_t* open, int64_t count) {
    if (!c) return ARC_E_INVALID;
    if (!open || count == 0) {
        if (!c->hopen.empty()) c->graph_valid = false;
        c->hopen.clear();
        c->src_dirty = true;
        return ARC_OK;
    }
    if (c->p.thin_approx) return fail(c, ARC_E_INVALID, "emission masks do not combine with thin_approx");
    const int64_t nbase = 12ll << (2 * c->p.l_base);
    if (count != (int64_t)c->hsrc.size() * nbase)
        return fail(c, ARC_E_INVALID, "mask has %lld entries, expected %lld (sources x 12*4^l_base)",
                    (long long)count, (long long)c->hsrc.size() * nbase);
    c->hopen.assign(open, open + count);
    c->src_dirty = true;
    c->graph_valid = false;
    return ARC_OK;
}

arc_status arc_set_thin_radii(arc_ctx* c, const double* radii, int nsrc) {
    if (!c) return ARC_E_INVALID;
    if (!c->p.thin_approx) return fail(c, ARC_E_STATE, "thin_approx is off");
    if (!radii || nsrc != (int)c->hsrc.size())
        return fail(c, ARC_E_INVALID, "need one radius per source (%d)", (int)c->hsrc.size());
    for (int i = 0; i < nsrc; ++i)
        if (!(radii[i] >= 0.0 && radii[i] <= 1e9))   // also keeps the FP32 copy finite
            return fail(c, ARC_E_INVALID, "radius %d invalid (need 0 <= R <= 1e9 cells)", i);
    arc_status st = upload_sources(c);
    if (st != ARC_OK) return st;
    if (c->nsrc_dev == 0) return ARC_OK;
    std::vector<float> h(c->nsrc_dev);
    for (int i = 0; i < c->nsrc_dev; ++i) h[i] = (float)radii[c->dev_ids[i]];
    CK(cudaMemcpyAsync(c->rthin, h.data(), h.size() * sizeof(float), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return ARC_OK;
}

arc_status arc_get_thin_radii(arc_ctx* c, double* radii, int nsrc, double* thin_photons) {
    if (!c) return ARC_E_INVALID;
    if (!c->p.thin_approx) return fail(c, ARC_E_STATE, "thin_approx is off");
    if (radii && nsrc != (int)c->hsrc.size())
        return fail(c, ARC_E_INVALID, "need room for one radius per source (%d)", (int)c->hsrc.size());
    std::vector<float> h(c->nsrc_dev);
    double thin = 0.0;
    if (c->nsrc_dev > 0 && !c->src_dirty)
        CK(cudaMemcpyAsync(h.data(), c->rthin, h.size() * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&thin, &c->scal->thin, sizeof thin, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (radii) {
        for (int i = 0; i < nsrc; ++i) radii[i] = 0.0;
        if (!c->src_dirty)
            for (int i = 0; i < c->nsrc_dev; ++i) radii[c->dev_ids[i]] = (double)h[i];
    }
    if (thin_photons) *thin_photons = c->traced ? thin * PHOT_UNIT * c->last_dt : 0.0;
    return ARC_OK;
}

arc_status arc_set_fault(arc_ctx* c, int64_t live_bias, double idle_timeout_s) {
    if (!c) return ARC_E_INVALID;
    if (live_bias < 0 || !(idle_timeout_s >= 1e-3 && idle_timeout_s <= 60.0))
        return fail(c, ARC_E_INVALID, "need live_bias >= 0 and 1 ms <= idle_timeout_s <= 60 s");
    c->fault_live_bias = live_bias;
    c->idle_timeout_ns = (unsigned long long)(idle_timeout_s * 1e9);
    c->graph_valid = false;
    return ARC_OK;
}

void arc_destroy(arc_ctx* c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    for (int i = 0; i < 4; ++i)
        if (c->ev[i]) cudaEventDestroy(c->ev[i]);
    void* ptrs[] = {c->nH, c->xHI, c->xHeI, c->xHeII, c->T, c->rec, c->gamma, c->heat,
                    c->dsrc, c->seeds, c->qdata, c->qseq, c->scal, c->absorbed_part, c->mlp, c->fb_list,
                    c->rthin, c->rnext, c->dopen};
    for (void* q : ptrs) dfree(q);
    if (c->own_stream) cudaStreamDestroy(c->stream);
    delete c;
}

}  // extern "C"
