// arc_trace.cu -- ray-tracing kernels of libarc (sm_103a).
//
//   k_prep       absorber optical depth per cell length, accumulators zeroed
//                (Sec. 2.1 step i; absorber densities from Sec. 2.3)
//   k_make_seeds 12 4^l_base / 4 work items per source (Sec. 2.1 step iii.a)
//   k_reset      work queue and counters
//   k_trace      persistent tracer: HEALPix pix2vec, cell-by-cell traversal,
//                Eq. (ion) absorption, split into 4 children, termination
//                (Sec. 2.1 step iii, Sec. 2.4)
//   k_finalize   per-group absorbed photons -> per-absorber photoionisation
//                and photoheating rates (Eq. ion, Sec. 2.8), FP64 partial sums
//                of the absorbed photons
//   k_budget     FP64 photon budget
//
// Design (GPU-first; differs from the paper's one-ray-per-core level loop):
// * one lane = one ray; a warp keeps the pending children of its splits on a
//   small deque in shared memory and always takes the newest (depth first), so
//   memory stays bounded by the tree depth instead of 48 4^l rays per level;
// * all sources run in one persistent launch: emitted work items are taken by
//   ticket from a static array ordered brightest first, and busy warps donate
//   the oldest (largest) pending subtrees to a bounded lock-free ring when
//   other warps are idle;
// * per segment a ray reads one 16-byte record of optical depth per cell
//   length (one per group) and adds the photons absorbed per group into the
//   cell with one vector atomic; the species split of Eq. (ion) depends only
//   on the cell's absorber densities, so it is applied once per cell in
//   k_finalize instead of per segment;
// * photon conservation is exact by construction: each segment moves exactly
//   D = N_before - N_after from the ray into the cell (Sterbenz-exact FP32
//   subtraction); the cell sums are FP32 and the rounding error of every
//   addition (TwoSum on the value the atomic returns) goes to an FP64 ledger;
// * a cell's record is one 32-byte sector: its optical depth per cell length
//   (read) followed by its absorbed photons (atomically added), so the read
//   brings into L2 the sector the atomic then updates;
// * geometry per segment is one FP32-pair addition: the distance to the next
//   plane of each axis is carried as a pair and advanced by |1/u| when that
//   plane is crossed, and the record index steps in the brick/Morton layout
//   (no per-segment recomputation from the source position).
#include <cuda_runtime.h>
#include <math.h>

#include "arc_internal.cuh"

namespace arc {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ long long ld_relaxed_s(const long long* p) {
    long long v;
    asm volatile("ld.relaxed.gpu.global.s64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long now_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// 128-bit atomic add returning the previous value (sm_90+ vector atomics)
__device__ __forceinline__ float4 atom_add_v4(float4* a, float4 v) {
    float4 o;
    asm volatile("atom.global.add.v4.f32 {%0,%1,%2,%3}, [%4], {%5,%6,%7,%8};"
                 : "=f"(o.x), "=f"(o.y), "=f"(o.z), "=f"(o.w)
                 : "l"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w));
    return o;
}
__device__ __forceinline__ float4 ldg_f4(const float4* p) { return __ldg(p); }

// rounding error of a + b (Knuth TwoSum, round-to-nearest throughout)
__device__ __forceinline__ float two_sum_err(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// rounding error of a + b for a, b >= 0: Fast2Sum on the larger and the
// smaller operand (exact, and the same value TwoSum gives, in five operations
// instead of six)
__device__ __forceinline__ float add_err_nonneg(float a, float b) {
    const float hi = fmaxf(a, b), lo = fminf(a, b);
    const float s = __fadd_rn(hi, lo);
    return __fsub_rn(lo, __fsub_rn(s, hi));
}
// Eq. (ion) for one group: the fraction a = 1 - exp(-tau) of the ray's
// photons is absorbed.  The ray carries its photons as an unevaluated pair
// Nh + Nl, so that it can lose exactly what the cell receives without the
// loss being rounded to a multiple of ulp(Nh) (which would make thin-cell
// deposits, a ~ 1e-5, wrong by ~6e-8/a).  The deposit is returned as the pair
// d + e and Nh + Nl + d + e is conserved up to ~2^-48 Nh per segment:
//   thin (a < 1/2): d = fl(Nh a), the ray subtracts d exactly;
//   thick:          the survivors fl(Nh e^-tau) are formed directly (no
//                   cancellation) and d + e is the exact difference.
//
// 1 - e^-tau for tau < ln 2 (the thin branch below): tau times the Taylor
// series of (1 - e^-tau) / tau to degree 9, by Horner in x = -tau with one FMA
// per term.  Truncation below tau^10 / 11! < 7e-10 relative, Horner rounding
// ~1e-7, so the per-segment error does not build up along rays that cross many
// cells of moderate depth (a hardware exponential's ~2e-6 did: 1e-4 after ~50
// such cells).  Photon conservation does not depend on it: the ray loses
// exactly what the cell receives.
__device__ __forceinline__ float thin_fraction(float tau) {
    const float x = -tau;
    float q = 1.0f / 3628800.0f;
    q = fmaf(q, x, 1.0f / 362880.0f);
    q = fmaf(q, x, 1.0f / 40320.0f);
    q = fmaf(q, x, 1.0f / 5040.0f);
    q = fmaf(q, x, 1.0f / 720.0f);
    q = fmaf(q, x, 1.0f / 120.0f);
    q = fmaf(q, x, 1.0f / 24.0f);
    q = fmaf(q, x, 1.0f / 6.0f);
    q = fmaf(q, x, 0.5f);
    q = fmaf(q, x, 1.0f);
    return tau * q;
}
// The branch is chosen on tau itself (a < 1/2 exactly when tau < ln 2), so a
// thick segment evaluates one exponential and a thin one none.
__device__ __forceinline__ void absorb(float& Nh, float& Nl, float tau, float& d, float& e) {
    if (tau < 0.69314718f) {
        const float a = thin_fraction(tau);
        d = __fmul_rn(Nh, a);
        e = 0.0f;
        const float s = __fsub_rn(Nh, d);                 // Fast2Sum(Nh, -d) = (s, r): d <= Nh / 2
        const float r = __fsub_rn(__fsub_rn(Nh, s), d);
        const float lo = __fadd_rn(Nl, r);
        Nh = __fadd_rn(s, lo);                            // renormalise (|lo| << |s|)
        Nl = __fsub_rn(lo, __fsub_rn(Nh, s));
    } else {
        // accurate exponential here: the hardware form's error grows with tau
        // (argument rounding), and through thick gas it would accumulate along
        // the ray
        const float Nn = __fmul_rn(Nh, expf(-tau));
        d = __fsub_rn(Nh, Nn);                            // Fast2Sum(Nh, -Nn) = (d, r): Nn <= Nh / 2
        const float r = __fsub_rn(__fsub_rn(Nh, d), Nn);
        e = __fadd_rn(r, Nl);
        Nh = Nn;
        Nl = 0.0f;
    }
}

// (Nh, Nl) <- Nh + lo as a normalised pair (|lo| within a few ulps of Nh)
__device__ __forceinline__ void fold_low(float& Nh, float& Nl, float lo) {
    const float s = __fadd_rn(Nh, lo);
    Nl = __fsub_rn(lo, __fsub_rn(s, Nh));
    Nh = s;
}

// Vector deposit of D = d + e into a cell's FP32 accumulator: the atomic
// returns the old value, from which the rounding error of old + d is
// recovered exactly (both are >= 0: Fast2Sum on the larger of the two); that
// error plus e, the part of the deposit below
// d's precision, is returned for the caller's rounding ledger.  The cell sums
// are then plain FP32 (relative error ~1e-7, far below the rates' needs) while
// the photon budget, cells plus ledger plus escapes, stays exact.
template <int NG>
__device__ __forceinline__ float deposit(float4* rec, uint64_t idx, float4 d, float4 e) {
    const float4 old = atom_add_v4(rec + 2 * idx + 1, d);
    float err = __fadd_rn(add_err_nonneg(old.x, d.x), e.x);
    if (NG > 1) err = __fadd_rn(err, __fadd_rn(add_err_nonneg(old.y, d.y), e.y));
    if (NG > 2) err = __fadd_rn(err, __fadd_rn(add_err_nonneg(old.z, d.z), e.z));
    if (NG > 3) err = __fadd_rn(err, __fadd_rn(add_err_nonneg(old.w, d.w), e.w));
    return err;
}

// ------------------------------------------------------------------ HEALPix
__device__ __forceinline__ uint32_t even_bits(uint32_t x) {
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0F0F0F0Fu;
    x = (x | (x >> 4)) & 0x00FF00FFu;
    x = (x | (x >> 8)) & 0x0000FFFFu;
    return x;
}

// ------------------------------------------------------------ pair arithmetic
// Unevaluated FP32 pairs hi + lo (~2^-44 relative) for the ray geometry.  The
// explicit _rn operations keep the compiler from contracting or reordering.
struct F2 {
    float h, l;
};
__device__ __forceinline__ F2 fast_two_sum(float a, float b) {   // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return F2{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ F2 f2_add(F2 a, F2 b) {
    const float s = __fadd_rn(a.h, b.h);
    const float e = __fadd_rn(two_sum_err(a.h, b.h), __fadd_rn(a.l, b.l));
    return fast_two_sum(s, e);
}
// a + b for a.h, b.h >= 0: the rounding error of the high parts by Fast2Sum
// on the larger of the two (the same value as f2_add's TwoSum)
__device__ __forceinline__ F2 f2_add_pos(F2 a, F2 b) {
    const float s = __fadd_rn(a.h, b.h);
    const float hi = fmaxf(a.h, b.h), lo = fminf(a.h, b.h);
    const float e = __fadd_rn(__fsub_rn(lo, __fsub_rn(s, hi)), __fadd_rn(a.l, b.l));
    return fast_two_sum(s, e);
}
__device__ __forceinline__ F2 f2_mul(F2 a, F2 b) {
    const float p = __fmul_rn(a.h, b.h);
    const float e = fmaf(a.h, b.l, fmaf(a.l, b.h, fmaf(a.h, b.h, -p)));
    return fast_two_sum(p, e);
}
__device__ __forceinline__ F2 f2_neg(F2 a) { return F2{-a.h, -a.l}; }
// num / den for integers exactly representable in FP32
__device__ __forceinline__ F2 f2_ratio(float num, float den) {
    const float h = __fdiv_rn(num, den);
    return F2{h, __fdiv_rn(fmaf(-h, den, num), den)};
}
__device__ __forceinline__ F2 f2_sqrt(F2 x) {
    const float h = __fsqrt_rn(x.h);
    if (h == 0.0f) return F2{0.0f, 0.0f};
    const float r = __fadd_rn(fmaf(-h, h, x.h), x.l);   // x - h^2 (the fma part is exact)
    return fast_two_sum(h, __fdiv_rn(r, __fadd_rn(h, h)));
}

// sin and cos of pi j / 64, j = -16..16, as pairs (sin h, sin l, cos h, cos l):
// each block of the tracer copies the table the host formed in FP64 (TraceArgs)
__shared__ float4 s_sincos[33];
__device__ __forceinline__ void load_sincos_table(const TraceArgs& A) {
    if (threadIdx.x < 33) s_sincos[threadIdx.x] = A.sincos[threadIdx.x];
    __syncthreads();
}

// Centre of nested pixel pix at level (nside = 2^level) as a unit vector of
// pairs (u[a] = hi + lo, ~1e-13).  The 12 base faces form three rows of four
// (north, equator, south); inside a face the pixel's (x, y) come from the
// even/odd bits of its index, which fix its ring (latitude) and its position
// along the ring (longitude).  Why pairs: a direction off by one FP32 ulp
// moves the ray ~t 1e-7 cells sideways, which behind optically thick cells
// (tens of optical depths per cell) changes the transmitted photons by
// ~1e-4.  Everything is FP32 arithmetic: z from its exact rational form,
// sin(theta) by a pair square root, and sin/cos of the longitude from the
// table above plus a short Taylor series in a remainder below pi / 128.
__device__ void healpix_dir(int level, uint64_t pix, F2 u[3]) {
    const int ns = 1 << level;
    const uint32_t face = (uint32_t)(pix >> (2 * level));
    const uint32_t ipf = (uint32_t)(pix & ((1ull << (2 * level)) - 1ull));
    const int ix = (int)even_bits(ipf), iy = (int)even_bits(ipf >> 1);
    const int row = (int)(face >> 2);
    const int ring = (row + 2) * ns - ix - iy - 1;      // 1 .. 4 ns - 1 from the north pole
    int nr, shift;
    F2 z, sth;
    if (ring < ns || ring > 3 * ns) {                   // polar caps: z = +-(1 - a), a = nr^2 / (3 ns^2)
        nr = ring < ns ? ring : 4 * ns - ring;
        const float f = __fdiv_rn((float)nr, (float)ns);   // exact (ns is a power of two)
        const F2 f2 = fast_two_sum(__fmul_rn(f, f), fmaf(f, f, -__fmul_rn(f, f)));
        const float ah = __fdiv_rn(f2.h, 3.0f);
        const F2 a = fast_two_sum(ah, __fdiv_rn(__fadd_rn(fmaf(-ah, 3.0f, f2.h), f2.l), 3.0f));
        const F2 one_minus = f2_add(F2{1.0f, 0.0f}, f2_neg(a));
        z = ring < ns ? one_minus : f2_neg(one_minus);
        sth = f2_sqrt(f2_mul(a, f2_add(F2{2.0f, 0.0f}, f2_neg(a))));   // a (2 - a)
        shift = 0;
    } else {                                            // belt: z = 2 (2 ns - ring) / (3 ns)
        nr = ns;
        z = f2_ratio((float)(2 * (2 * ns - ring)), (float)(3 * ns));
        sth = f2_sqrt(f2_add(F2{1.0f, 0.0f}, f2_neg(f2_mul(z, z))));   // 1 - z^2
        shift = (ring - ns) & 1;
    }
    const int lon = 2 * (int)(face & 3u) + (row == 1 ? 0 : 1);
    int jp = (lon * nr + ix - iy + 1 + shift) >> 1;     // numerator is always even
    if (jp > 4 * ns) jp -= 4 * ns;
    if (jp < 1) jp += 4 * ns;
    // longitude / pi = m / (4 nr), reduced exactly (in integers) to the
    // nearest multiple of 1/2 (k) plus q = mq / (4 nr), |q| <= 1/4, and q to
    // the nearest multiple of 1/64 (j) plus d = dn / (64 nr), |d| <= 1/128
    const int m = 2 * jp - shift - 1;
    const int half = 2 * nr;
    const int k = (m + nr) / half;                      // m >= 0
    const int mq = m - k * half;                        // -nr .. nr
    const int j = (int)rintf(__fdiv_rn((float)(16 * mq), (float)nr));
    const F2 d = f2_ratio((float)(16 * mq - j * nr), (float)(64 * nr));
    const F2 th = f2_mul(d, F2{3.14159274101257324f, -8.74227766e-8f});   // pi d
    const float t2 = __fmul_rn(th.h, th.h);
    // sin(th) = th - th^3/6 + th^5/120, cos(th) = 1 - th^2/2 + th^4/24 - th^6/720
    // (|th| < 0.025: the next terms are below 2e-15)
    const F2 sb = fast_two_sum(th.h, __fadd_rn(th.l, __fmul_rn(__fmul_rn(th.h, t2),
                                                               fmaf(t2, 1.0f / 120.0f, -1.0f / 6.0f))));
    const float t2l = fmaf(th.h, th.h, -t2) + 2.0f * th.h * th.l;   // th^2 = t2 + t2l
    const F2 c0 = fast_two_sum(1.0f, -0.5f * t2);
    const F2 cb = fast_two_sum(c0.h, __fadd_rn(c0.l, fmaf(-0.5f, t2l,
                                                          __fmul_rn(__fmul_rn(t2, t2),
                                                                    fmaf(t2, -1.0f / 720.0f, 1.0f / 24.0f)))));
    const float4 tab = s_sincos[j + 16];
    const F2 sa{tab.x, tab.y}, ca{tab.z, tab.w};
    const F2 s0 = f2_add(f2_mul(sa, cb), f2_mul(ca, sb));            // sin(pi q)
    const F2 c0q = f2_add(f2_mul(ca, cb), f2_neg(f2_mul(sa, sb)));   // cos(pi q)
    F2 sp, cp;
    switch (k & 3) {
        case 0: sp = s0; cp = c0q; break;
        case 1: sp = c0q; cp = f2_neg(s0); break;
        case 2: sp = f2_neg(s0); cp = f2_neg(c0q); break;
        default: sp = f2_neg(c0q); cp = s0; break;
    }
    u[0] = f2_mul(sth, cp);
    u[1] = f2_mul(sth, sp);
    u[2] = z;
}

// 1/u as a pair ih + il: ih the FP32 reciprocal of the high part, il from the
// residual 1 - (uh + ul) ih.  A zero component gives ih = +-inf, il = 0.
__device__ __forceinline__ void inv_pair(F2 u, float& ih, float& il) {
    ih = __frcp_rn(u.h);
    il = (u.h == 0.0f) ? 0.0f : __fmul_rn(fmaf(-u.l, ih, fmaf(-u.h, ih, 1.0f)), ih);
}

// floor(o + r u) for the start cell, with the origin o = oh + ol and u pairs:
// the sum is formed as a pair and the floor taken of its exact value
__device__ __forceinline__ int start_cell(float oh, float ol, float r, F2 u) {
    const F2 p = f2_mul(F2{r, 0.0f}, u);
    const float sh = __fadd_rn(oh, p.h);
    const float low = __fadd_rn(__fadd_rn(two_sum_err(oh, p.h), p.l), ol);
    float c = floorf(sh);
    if (sh == c && low < 0.0f) c -= 1.0f;
    else if (low > 0.0f && low >= __fsub_rn(c + 1.0f, sh)) c += 1.0f;
    return (int)c;
}

// ------------------------------------------------------------------ work queue
// Bounded multi-producer multi-consumer ring with one sequence word per slot:
// the slot of position p is free for a producer when seq == p and holds data
// for a consumer when seq == p + 1; a consumer frees it with seq = p + cap.
// A warp reserves a run of consecutive slots with one CAS on tail (push) or
// head (pop) after checking every slot of the run, so neither side ever waits
// on another thread: the operations are lock-free and only retry the CAS.

// Push the entries held by lanes 0..cnt-1 (cnt <= 32).  All lanes call.
// A mandatory push (the deque overflows) retries up to 2^20 times and flags
// ERR_QUEUE_FULL / ERR_CAS_SPIN on failure; an optional one (sharing work
// with idle warps) gives up quietly after a few lost races.  Returns whether
// the entries were pushed.
__device__ bool q_push_warp(const TraceArgs& A, const Entry& e, unsigned cnt, int lane,
                            bool mandatory) {
    if (cnt == 0) return true;
    const int tries = mandatory ? (1 << 20) : 16;
    for (int it = 0; it < tries; ++it) {
        unsigned long long pos = 0;
        if (lane == 0) pos = ld_relaxed(A.qtail);
        pos = __shfl_sync(FULL, pos, 0);
        long long dif = 0;
        if ((unsigned)lane < cnt) {
            const unsigned long long p = pos + (unsigned long long)lane;
            dif = (long long)(ld_acquire(&A.qseq[p & A.qmask]) - p);
        }
        const unsigned full = __ballot_sync(FULL, dif < 0);
        if (full) {
            if (mandatory && lane == 0) atomicOr(A.status, ERR_QUEUE_FULL);
            return false;
        }
        if (__ballot_sync(FULL, dif > 0)) continue;   // stale tail: re-read
        unsigned long long got = 0;
        if (lane == 0) got = atomicCAS(A.qtail, pos, pos + cnt);
        got = __shfl_sync(FULL, got, 0);
        if (got != pos) {
            __nanosleep(64u << (it & 3));   // lost the race to another producer
            continue;
        }
        {
            if ((unsigned)lane < cnt) {
                const unsigned long long p = pos + (unsigned long long)lane;
                float4* d = reinterpret_cast<float4*>(&A.qdata[p & A.qmask]);
                __stcg(d, *reinterpret_cast<const float4*>(&e));
                __stcg(d + 1, e.N);
                st_release(&A.qseq[p & A.qmask], p + 1);
            }
            return true;
        }
    }
    if (mandatory && lane == 0) atomicOr(A.status, ERR_CAS_SPIN);
    return false;
}

// Pop up to `want` (<= 32) entries; lane i < (returned count) receives entry i.
// All lanes call.  Returns 0 when nothing is published at the head, or after a
// few lost races with other consumers (each loss is another warp's progress;
// the caller polls again later).
__device__ int q_pop_warp(const TraceArgs& A, Entry& e, int want, int lane) {
    for (int it = 0; it < 32; ++it) {
        unsigned long long pos = 0;
        if (lane == 0) pos = ld_relaxed(A.qhead);
        pos = __shfl_sync(FULL, pos, 0);
        bool ready = false;
        long long dif = -1;
        if (lane < want) {
            const unsigned long long p = pos + (unsigned long long)lane;
            dif = (long long)(ld_acquire(&A.qseq[p & A.qmask]) - (p + 1));
            ready = dif == 0;
        }
        const unsigned rm = __ballot_sync(FULL, ready);
        const int c = (rm == FULL) ? 32 : (__ffs(~rm) - 1);   // consecutive ready slots from the head
        if (c == 0) {
            // slot at head not published: empty, or head is stale (dif > 0)
            const int stale = __shfl_sync(FULL, (int)(dif > 0), 0);
            if (stale) continue;
            return 0;
        }
        unsigned long long got = 0;
        if (lane == 0) got = atomicCAS(A.qhead, pos, pos + (unsigned long long)c);
        got = __shfl_sync(FULL, got, 0);
        if (got != pos) {
            __nanosleep(64u << (it & 3));   // lost the race: back off a little
            continue;
        }
        {
            if (lane < c) {
                const unsigned long long p = pos + (unsigned long long)lane;
                const float4* d = reinterpret_cast<const float4*>(&A.qdata[p & A.qmask]);
                const float4 x = __ldcg(d);
                const float4 y = __ldcg(d + 1);
                *reinterpret_cast<float4*>(&e) = x;
                e.N = y;
                st_release(&A.qseq[p & A.qmask], p + A.qmask + 1);
            }
            return c;
        }
    }
    return 0;
}

// ------------------------------------------------------------------ ray state
// EV_BLOCK: an emitted ray whose direction the source's mask blocks (Sec. 2.2)
enum : int { EV_NONE = 0, EV_SPLIT = 1, EV_ESC = 2, EV_TERM = 3, EV_BLOCK = 4 };

// Ray geometry (Sec. 2.4: the ray crosses the grid cell by cell).  The
// distance from the source to the next X, Y and Z plane is carried as an
// unevaluated FP32 pair (~2^-44 relative) and advanced by |1/u| (a pair as
// well) when that plane is crossed: one pair addition per segment instead of
// three plane-distance products.  With plain FP32 a crossing distance t would
// be off by ~t 2^-24 cells, and behind cells of tens of optical depths that
// moves ~1e-4 of the photons.  The ray's source, level and pixel are needed
// only at events; they live in shared memory, one slot per thread, which keeps
// them out of the registers of the segment loop.
struct Ray {
    float tx, tlx, ty, tly, tz, tlz;   // next plane per axis (hi, lo); u = 0: hi = +inf and lo
                                        // holds the fixed in-cell coordinate o - c
    float ix, iy, iz;      // 1/u per axis (+-inf for u = 0), high parts
    float ilx, ily, ilz;   // low parts of 1/u
    int cx, cy, cz;        // current cell
    float r, rl;           // distance travelled (hi + lo)
    float rstop, thr;
    float4 N;              // photons per group (high part)
    float4 Nl;             // low part: the photons are N + Nl
    float4 kap;            // optical depth per cell length of the current cell
    uint32_t idx;          // brick-cell index of the current cell
    uint32_t visits;
    float cthr;            // thin radius: group-0 photons at optical depth 0.1 of this
                           // ray's share; 0 once reached (or the group is empty)
};
struct RayId {
    uint64_t pix;
    uint32_t src;
    int level;
};
__shared__ RayId s_id[256];   // per thread of the block (k_trace blocks have <= 256 threads)

// distance to the next plane on one axis from the origin oh + ol, as a pair
// th + tl: (P - oh - ol)(ih + il) with P - oh exact (TwoSum) and the product's
// rounding error recovered by FMA.  u > 0 (ih > 0): plane c + 1; u < 0: plane
// c; u = 0 (ih infinite): +inf
__device__ __forceinline__ float next_plane_t(int c, float oh, float ol, float ih, float il, float& tl) {
    const float P = (float)(c + (ih > 0.0f ? 1 : 0));
    const float ah = __fsub_rn(P, oh);
    const float al = __fsub_rn(two_sum_err(P, -oh), ol);
    const float th = __fmul_rn(ah, ih);
    const F2 t = fast_two_sum(th, fmaf(al, ih, fmaf(ah, il, fmaf(ah, ih, -th))));
    const bool par = fabsf(ih) == INFINITY;
    tl = par ? 0.0f : t.l;
    return par ? INFINITY : t.h;
}

// Start child k of entry e in this lane.  Returns EV_ESC if the child starts
// outside the box (it then carries its photons straight to the escape ledger).
// The EXT variant (emission masks, Sec. 2.2; optically thin radius, Sec. 2.6)
// also returns EV_BLOCK for an emitted ray the source's mask blocks, and
// EV_SPLIT for a ray that starts at or beyond its split distance (rays
// launched at the thin radius): it splits at once without tracing a cell.
template <bool EXT>
__device__ __forceinline__ int start_ray(const TraceArgs& A, const Entry& e, int k, Ray& R) {
    const int level = key_level(e.key);
    const uint64_t pix = key_pixbase(e.key) + (uint64_t)k;
    RayId& id = s_id[threadIdx.x];
    id.pix = pix;
    id.src = e.src;
    id.level = level;
    R.r = e.r;
    R.rl = 0.0f;
    R.N = e.N;
    R.Nl = make_float4(0.f, 0.f, 0.f, 0.f);
    R.visits = 0;
    const SourceDev* S = &A.src[e.src];
    const float4 pt = __ldg(&S->pos_thr);
    const float4 pl = __ldg(&S->pos_lo);
    R.thr = ldexpf(pt.w, -2 * (level - A.l_base));
    R.rstop = (level < A.l_max) ? A.rsplit[level] : INFINITY;
    if (EXT) {
        const float c = ldexpf(pl.w, -2 * (level - A.l_base));
        R.cthr = (A.rnext != nullptr && R.N.x > c) ? c : 0.0f;
        if (A.open != nullptr && level == A.l_base && A.open[(size_t)e.src * A.nbase + pix] == 0) {
            R.cthr = 0.0f;
            return EV_BLOCK;
        }
    }
    F2 u[3];
    healpix_dir(level, pix, u);
    inv_pair(u[0], R.ix, R.ilx);
    inv_pair(u[1], R.iy, R.ily);
    inv_pair(u[2], R.iz, R.ilz);
    R.cx = start_cell(pt.x, pl.x, R.r, u[0]);
    R.cy = start_cell(pt.y, pl.y, R.r, u[1]);
    R.cz = start_cell(pt.z, pl.z, R.r, u[2]);
    const int n = A.n;
    if (R.cx < 0 || R.cx >= n || R.cy < 0 || R.cy >= n || R.cz < 0 || R.cz >= n) return EV_ESC;
    float tl;
    R.tx = next_plane_t(R.cx, pt.x, pl.x, R.ix, R.ilx, tl);
    R.tlx = (R.tx == INFINITY) ? __fadd_rn(__fsub_rn(pt.x, (float)R.cx), pl.x) : tl;
    R.ty = next_plane_t(R.cy, pt.y, pl.y, R.iy, R.ily, tl);
    R.tly = (R.ty == INFINITY) ? __fadd_rn(__fsub_rn(pt.y, (float)R.cy), pl.y) : tl;
    R.tz = next_plane_t(R.cz, pt.z, pl.z, R.iz, R.ilz, tl);
    R.tlz = (R.tz == INFINITY) ? __fadd_rn(__fsub_rn(pt.z, (float)R.cz), pl.z) : tl;
    if (EXT && R.r >= R.rstop) return EV_SPLIT;
    R.idx = (uint32_t)brick_index(R.cx, R.cy, R.cz, A.nb);
    R.kap = ldg_f4(&A.kappa[2 * (size_t)R.idx]);
    return EV_NONE;
}

// One cell segment (Sec. 2.4): to the nearest X/Y/Z boundary or the split
// distance, Eq. (ion) absorption in each of the NG groups, then step.  The
// next cell's record is loaded before the current cell's deposit is issued, so
// the load and the atomic round trip overlap.
template <int NG, bool REC, bool EXT>
__device__ __forceinline__ int segment(const TraceArgs& A, Ray& R, float& rerr) {
    // nearest plane; ties go to the lowest axis (x, y, z), as in the step below
    const bool ax = R.tx <= R.ty && R.tx <= R.tz;
    const bool ay = !ax && R.ty <= R.tz;
    const float t = ax ? R.tx : (ay ? R.ty : R.tz);
    const float tl = ax ? R.tlx : (ay ? R.tly : R.tlz);
    // split where r_split <= t exactly (r_split is an FP32 value, t = hi + lo)
    const bool split = R.rstop < t || (R.rstop == t && tl >= 0.0f);
    const float r1 = split ? R.rstop : t;
    const float r1l = split ? 0.0f : tl;
    const float ds = fmaxf(__fadd_rn(__fsub_rn(r1, R.r), __fsub_rn(r1l, R.rl)), 0.0f);
    const uint32_t idx = R.idx;
    const float4 kap = R.kap;
    const float4 Nh0 = R.N, Nl0 = R.Nl;
    float4 D = make_float4(0.f, 0.f, 0.f, 0.f), E = make_float4(0.f, 0.f, 0.f, 0.f);
    absorb(R.N.x, R.Nl.x, kap.x * ds, D.x, E.x);
    if (NG > 1) absorb(R.N.y, R.Nl.y, kap.y * ds, D.y, E.y);
    if (NG > 2) absorb(R.N.z, R.Nl.z, kap.z * ds, D.z, E.z);
    if (NG > 3) absorb(R.N.w, R.Nl.w, kap.w * ds, D.w, E.w);
    if (EXT && R.cthr > 0.0f && R.N.x <= R.cthr) {
        // Sec. 2.6: the group-0 optical depth from the ray's start reaches 0.1
        // inside this segment, at r + ln(N_in / N_0.1) / kappa_0
        float ts = r1;
        if (kap.x > 0.0f) ts = fminf(fmaxf(R.r + logf(Nh0.x / R.cthr) / kap.x, R.r), r1);
        atomicMin(reinterpret_cast<int*>(A.rnext) + s_id[threadIdx.x].src, __float_as_int(ts));
        R.cthr = 0.0f;
    }
    float sumN = R.N.x;
    if (NG > 1) sumN += R.N.y;
    if (NG > 2) sumN += R.N.z;
    if (NG > 3) sumN += R.N.w;
    const bool term = sumN < R.thr;
    const float4 Dabs = D;   // this segment's Eq. (ion) absorption
    if (term) {
        // below threshold: every remaining photon stays in this cell
        D = make_float4(Nh0.x, NG > 1 ? Nh0.y : 0.f, NG > 2 ? Nh0.z : 0.f, NG > 3 ? Nh0.w : 0.f);
        E = make_float4(Nl0.x, NG > 1 ? Nl0.y : 0.f, NG > 2 ? Nl0.z : 0.f, NG > 3 ? Nl0.w : 0.f);
        R.N = make_float4(0.f, 0.f, 0.f, 0.f);
        R.Nl = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (REC) R.visits++;   // per-ray records only
    // Sec. 2.5, Eq. (correction): near a face of the cell (midpoint closer than
    // half the pixel width) the fraction 1 - f_c of the photons absorbed here
    // goes to the neighbour across that face (Eq. correction2, as photons split
    // over the neighbour's own absorbers in k_finalize).  The moved part is
    // taken from the absorbed part only; at a termination the residual stays.
    uint32_t nidx = 0;
    float4 Dn = make_float4(0.f, 0.f, 0.f, 0.f);
    bool corr = false;
    if (A.geo_corr && ds > 0.0f) {
        // in-cell coordinates of the midpoint from the pair distances: along an
        // axis with u != 0 the far face (the next plane) lies (t_a - r_m)|u_a|
        // away, to FP32 precision of that sub-cell distance; along u = 0 the
        // coordinate is fixed
        const F2 rm2 = f2_add(F2{R.r, R.rl}, F2{r1, r1l});
        const float rm = 0.5f * rm2.h;
        const F2 mrm = F2{-0.5f * rm2.h, -0.5f * rm2.l};
        float f[3];
        {
            const float th[3] = {R.tx, R.ty, R.tz}, tlo[3] = {R.tlx, R.tly, R.tlz};
            const float ih[3] = {R.ix, R.iy, R.iz};
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                if (th[a] == INFINITY) {
                    f[a] = tlo[a];
                } else {
                    const F2 q = f2_add(F2{th[a], tlo[a]}, mrm);
                    const float dn = __fdiv_rn(__fadd_rn(q.h, q.l), fabsf(ih[a]));
                    f[a] = ih[a] > 0.0f ? __fsub_rn(1.0f, dn) : dn;
                }
            }
        }
        float dmin = INFINITY;
        int nax = 0, nside = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {   // faces -x, +x, -y, +y, -z, +z; ties to the first
            if (f[a] < dmin) { dmin = f[a]; nax = a; nside = -1; }
            if (1.0f - f[a] < dmin) { dmin = 1.0f - f[a]; nax = a; nside = 1; }
        }
        dmin = fmaxf(dmin, 0.0f);
        const float lpix = rm * A.pixw[s_id[threadIdx.x].level];
        int nb[3] = {R.cx, R.cy, R.cz};
        nb[nax] += nside;
        if (dmin < 0.5f * lpix && nb[nax] >= 0 && nb[nax] < A.n) {
            const float fc = 0.5f + __fdiv_rn(dmin, lpix);
            nidx = (uint32_t)brick_index(nb[0], nb[1], nb[2], A.nb);
            const float4 nk = ldg_f4(&A.kappa[2 * (size_t)nidx]);
            // moved photons per group (none where the neighbour has no absorber);
            // d - moved is exact because moved <= d / 2
            const float g = 1.0f - fc;
            Dn.x = nk.x > 0.f ? __fmul_rn(g, Dabs.x) : 0.f;
            if (NG > 1) Dn.y = nk.y > 0.f ? __fmul_rn(g, Dabs.y) : 0.f;
            if (NG > 2) Dn.z = nk.z > 0.f ? __fmul_rn(g, Dabs.z) : 0.f;
            if (NG > 3) Dn.w = nk.w > 0.f ? __fmul_rn(g, Dabs.w) : 0.f;
            corr = Dn.x != 0.f || Dn.y != 0.f || Dn.z != 0.f || Dn.w != 0.f;
        }
    }
    R.r = r1;
    R.rl = r1l;
    int ev = term ? EV_TERM : (split ? EV_SPLIT : EV_NONE);
    if (ev == EV_NONE) {
        // step across the nearest face (ties to the lowest axis): the cell, that
        // axis's next-plane distance (+ |1/u|) and the record index (that axis's
        // Morton bits inside the 8^3 brick, carrying or borrowing into the brick
        // index)
        const float ih = ax ? R.ix : (ay ? R.iy : R.iz);
        const float il = ax ? R.ilx : (ay ? R.ily : R.ilz);
        const bool up = ih > 0.0f;
        const F2 tn = f2_add_pos(F2{t, tl}, F2{fabsf(ih), up ? il : -il});
        const int c = (ax ? R.cx : (ay ? R.cy : R.cz)) + (up ? 1 : -1);
        const uint32_t mk = ax ? 0x124u : (ay ? 0x92u : 0x49u);
        const uint32_t bs = ax ? A.bstride_x : (ay ? A.bstride_y : 512u);
        const uint32_t m = R.idx;
        const uint32_t mm = up ? (((m | ~mk) + 1u) & mk) : (((m & mk) - 1u) & mk);
        uint32_t ni = (m & ~mk) | mm;
        if (up && mm == 0u) ni += bs;
        if (!up && mm == mk) ni -= bs;
        if (ax) {
            R.cx = c;
            R.tx = tn.h;
            R.tlx = tn.l;
        } else if (ay) {
            R.cy = c;
            R.ty = tn.h;
            R.tly = tn.l;
        } else {
            R.cz = c;
            R.tz = tn.h;
            R.tlz = tn.l;
        }
        if ((unsigned)c >= (unsigned)A.n) {
            ev = EV_ESC;
        } else {
            R.idx = ni;
            R.kap = ldg_f4(&A.kappa[2 * (size_t)ni]);
        }
    }
    if (corr) {
        D.x = __fsub_rn(D.x, Dn.x);   // exact: Dn <= D / 2
        D.y = __fsub_rn(D.y, Dn.y);
        D.z = __fsub_rn(D.z, Dn.z);
        D.w = __fsub_rn(D.w, Dn.w);
        rerr = __fadd_rn(rerr, deposit<NG>(A.acc, nidx, Dn, make_float4(0.f, 0.f, 0.f, 0.f)));
    }
    // unconditional: a segment that deposits nothing (an empty cell) adds zeros,
    // which leaves the cell and the ledger as they were
    rerr = __fadd_rn(rerr, deposit<NG>(A.acc, idx, D, E));
    return ev;
}

// per-warp tallies of one launch (shared memory)
struct WarpTally {
    unsigned long long nrays, nsplit, nterm, nesc, ndon;
    double esc;                // photons that left the box
    long long live_delta;      // rays created minus finished, not yet flushed
    unsigned maxlev;
};

#ifndef ARC_SEG_BATCH
#define ARC_SEG_BATCH 32   // measured on the 256^3 field, 1000 sources (this tracer, lane ledgers in
                           // shared memory): 12 -> 54.2, 16 -> 58.2, 24 -> 61.0, 32 -> 61.6,
                           // 48 -> 60.0, 64 -> 59.5 Gsegments/s
#endif
#ifndef ARC_REFILL_IDLE
#define ARC_REFILL_IDLE 16
#endif
constexpr int SEG_BATCH = ARC_SEG_BATCH;   // segments per lane between warp event rounds
constexpr int HEARTBEAT_EVERY = 1024; // event rounds between progress signals

#ifndef ARC_TRACE_MIN_BLOCKS
#define ARC_TRACE_MIN_BLOCKS 3   // resident 256-thread blocks per SM the registers must allow
                                 // (3: 80 registers, 24 warps/SM; measured 16 % faster than 2
                                 // blocks without spills, and faster than 4)
#endif
template <int NG, bool REC, bool EXT>
__global__ void __launch_bounds__(256, ARC_TRACE_MIN_BLOCKS) k_trace(const TraceArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const unsigned cap = 1u << A.stack_log2;       // >= 64, so one round's pushes fit in half
    const unsigned cmask = cap - 1u;
    Entry* stack = reinterpret_cast<Entry*>(smem_raw) + (size_t)wib * cap;
    const unsigned lt_mask = (1u << lane) - 1u;

    // deque [bot, top) of pending work items, indices modulo cap (warp-uniform)
    unsigned bot = 0, top = 0;
    // per-warp tallies live in shared memory (written by lane 0, escapes by
    // shared FP64 atomics) so that they do not hold registers in every lane
    __shared__ WarpTally tally_all[8];
    WarpTally& W = tally_all[wib];
    if (lane == 0) W = WarpTally{};
    load_sincos_table(A);   // also orders the tallies' initialisation
    // per-lane segment count and rounding ledger (photons the FP32 cell sums
    // rounded away, exact) in shared memory: updated once per batch, they hold
    // no registers in the segment loop
    __shared__ double s_round[256];
    __shared__ unsigned s_nseg[256];
    s_round[threadIdx.x] = 0.0;
    s_nseg[threadIdx.x] = 0u;
    unsigned round = 0;

    Ray R;
    bool active = false;
    int ev = EV_NONE;

    auto flush_live = [&]() {
        if (lane == 0 && W.live_delta != 0) {
            atomicAdd(reinterpret_cast<unsigned long long*>(A.live), (unsigned long long)W.live_delta);
            W.live_delta = 0;
        }
    };
    // move the oldest `cnt` items of the deque to the global ring (all lanes)
    auto donate = [&](unsigned cnt, bool mandatory) {
        flush_live();   // rays made visible to other warps must be counted first
        __syncwarp();
        while (cnt > 0) {
            const unsigned chunk = cnt < 32u ? cnt : 32u;
            Entry e;
            if ((unsigned)lane < chunk) e = stack[(bot + lane) & cmask];
            __syncwarp();
            if (!q_push_warp(A, e, chunk, lane, mandatory)) break;   // not pushed: keep them here
            bot += chunk;
            if (lane == 0) W.ndon += chunk;
            cnt -= chunk;
        }
    };
    // place up to `want` global items on the (empty) deque: donated subtrees
    // first, then emitted items by ticket; returns the count (all lanes)
    auto acquire = [&](int want) -> int {
        Entry e;
        const int c = q_pop_warp(A, e, want, lane);
        if (c > 0) {
            if (lane < c) stack[(top + lane) & cmask] = e;
            __syncwarp();
            return c;
        }
        unsigned t0 = 0;
        int got = 0;
        if (lane == 0 && ld_relaxed_u32(A.seed_head) < (unsigned)A.nseeds) {
            t0 = atomicAdd(A.seed_head, (unsigned)want);
            const int avail = A.nseeds - (int)t0;
            got = avail <= 0 ? 0 : (avail < want ? avail : want);
        }
        got = __shfl_sync(FULL, got, 0);
        t0 = __shfl_sync(FULL, t0, 0);
        if (lane < got) stack[(top + lane) & cmask] = A.seeds[t0 + lane];
        __syncwarp();
        return got;
    };

    bool done = false;
    while (!done) {
        // ---------------------------------------------------------------- refill
        unsigned idle = __ballot_sync(FULL, !active);
        if (idle) {
            const int nidle = __popc(idle);
            if (top == bot && (idle == FULL || (nidle >= ARC_REFILL_IDLE && (round & 3) == 0))) {
                int got = acquire((nidle + 3) >> 2);
                if (got == 0 && idle == FULL) {
                    // nothing anywhere for now: wait (bounded) for donations or the end
                    flush_live();
                    __syncwarp();
                    if (lane == 0) atomicAdd(A.n_idle, 1);
                    unsigned long long t_last = now_ns();
                    unsigned hb_last = ld_relaxed_u32(A.heartbeat);
                    long long live_last = ld_relaxed_s(A.live);
                    unsigned sleep = 32;
                    int result = 0;   // 1 work, 2 finished, 3 gave up
                    // bounded: 10 s (idle_timeout_ns) or 2^24 polls without any sign of
                    // progress elsewhere end the wait with an error status
                    for (unsigned poll = 0; poll < (1u << 24); ++poll) {
                        got = acquire(8);
                        if (got > 0) {
                            result = 1;
                            break;
                        }
                        int r = 0, progressed = 0;
                        if (lane == 0) {
                            const long long lv = ld_relaxed_s(A.live);
                            const unsigned hb = ld_relaxed_u32(A.heartbeat);
                            const unsigned long long tn = now_ns();
                            if (lv == 0) {
                                r = 2;
                            } else if (ld_relaxed_u32(A.status) & (ERR_TIMEOUT | ERR_CAS_SPIN)) {
                                r = 3;
                            } else if (hb != hb_last || lv != live_last) {
                                hb_last = hb;
                                live_last = lv;
                                t_last = tn;
                                progressed = 1;
                            } else if (tn - t_last > A.idle_timeout_ns) {
                                atomicOr(A.status, ERR_TIMEOUT);
                                r = 3;
                            }
                        }
                        r = __shfl_sync(FULL, r, 0);
                        if (r) {
                            result = r;
                            break;
                        }
                        if (__shfl_sync(FULL, progressed, 0)) poll = 0;
                        __nanosleep(sleep);
                        if (sleep < 2048) sleep <<= 1;
                    }
                    if (result == 0) {
                        if (lane == 0) atomicOr(A.status, ERR_TIMEOUT);
                        result = 3;
                    }
                    if (lane == 0) atomicSub(A.n_idle, 1);
                    if (result != 1) {
                        done = true;
                        break;
                    }
                }
                top += (unsigned)got;
            }
            // hand the children of the newest items to idle lanes (depth first):
            // each lane notes its item's slot and child, and all lanes that took
            // one start their rays together after the loop (a ray start is a
            // few hundred instructions: started item by item, only the 1-4
            // lanes of that item would be active).  Slots given up here are not
            // reused before the event phase, so the items are still in place.
            int take_slot = -1, take_k = 0;
            while (idle != 0 && top != bot) {
                const unsigned slot = (top - 1) & cmask;
                const uint64_t key = stack[slot].key;
                const int k0 = key_k(key);
                const int avail = 4 - k0;
                const int rank = __popc(idle & lt_mask);
                const bool mine = ((idle >> lane) & 1u) && rank < avail;
                const unsigned taken = __ballot_sync(FULL, mine);
                if (mine) {
                    take_slot = (int)slot;
                    take_k = k0 + rank;
                }
                if (lane == 0) {
                    W.nrays += (unsigned)__popc(taken);
                    W.maxlev = max(W.maxlev, (unsigned)key_level(key));
                }
                idle &= ~taken;
                __syncwarp();
                const int ntake = __popc(taken);
                if (ntake >= avail) {
                    top -= 1;
                } else if (lane == 0) {
                    stack[slot].key = make_key(key_pixbase(key), key_level(key), k0 + ntake);
                }
                __syncwarp();
            }
            if (take_slot >= 0) {
                ev = start_ray<EXT>(A, stack[take_slot], take_k, R);
                active = true;
            }
        }

        // ------------------------------------------------------------ trace
        if (active && ev == EV_NONE) {
            float rerr = 0.0f;   // rounding ledger of this batch (a few ulps of its deposits)
            int it = 0;
#pragma unroll 1
            for (; it < SEG_BATCH; ++it) {
                ev = segment<NG, REC, EXT>(A, R, rerr);
                if (ev != EV_NONE) break;
            }
            s_nseg[threadIdx.x] += (unsigned)(it < SEG_BATCH ? it + 1 : SEG_BATCH);
            s_round[threadIdx.x] += (double)rerr;
        }

        // ------------------------------------------------------------ events
        const bool has_ev = active && ev != EV_NONE;
        const unsigned evm = __ballot_sync(FULL, has_ev);
        if (evm) {
            // per-ray records (test aid)
            if (REC && A.recs != nullptr) {
                unsigned long long base = 0;
                if (lane == 0) base = atomicAdd(A.nrec, (unsigned long long)__popc(evm));
                base = __shfl_sync(FULL, base, 0);
                if (has_ev) {
                    const unsigned long long slot = base + __popc(evm & lt_mask);
                    if (slot < A.rec_cap) {
                        arc_ray_rec q;
                        const RayId& id = s_id[threadIdx.x];
                        q.src = A.src[id.src].id;
                        q.level = (uint8_t)id.level;
                        q.end = (uint8_t)ev;
                        q.pad = 0;
                        q.pix = id.pix;
                        q.visits = R.visits;
                        q.r1 = R.r;
                        A.recs[slot] = q;
                    } else {
                        atomicOr(A.status, ERR_RECORDS);
                    }
                }
            }
            const bool is_split = has_ev && ev == EV_SPLIT;
            // Sec. 2.6: a ray that ends (escape, threshold) before its group-0
            // optical depth reaches 0.1 offers its whole length
            if (EXT && has_ev && !is_split && R.cthr > 0.0f)
                atomicMin(reinterpret_cast<int*>(A.rnext) + s_id[threadIdx.x].src, __float_as_int(R.r));
            if (has_ev && !is_split) {
                if (ev == EV_ESC) {
                    atomicAdd(&W.esc, ((double)R.N.x + (double)R.Nl.x) + ((double)R.N.y + (double)R.Nl.y) +
                                          ((double)R.N.z + (double)R.Nl.z) +
                                          (NG > 3 ? ((double)R.N.w + (double)R.Nl.w) : 0.0));
                }
            }
            const unsigned escm = __ballot_sync(FULL, has_ev && !is_split && ev == EV_ESC);
            if (has_ev && !is_split) {
                active = false;
                ev = EV_NONE;
            }
            const unsigned sm = __ballot_sync(FULL, is_split);
            const unsigned em = evm & ~sm;
            if (lane == 0) {
                W.live_delta += 3 * (long long)__popc(sm) - (long long)__popc(em);
                W.nesc += (unsigned)__popc(escm);
                W.nterm += (unsigned)__popc(em & ~escm);
                W.nsplit += (unsigned)__popc(sm);
                W.nrays += (unsigned)__popc(sm);
            }
            if (sm) {
                // make room: donate the oldest items if this round's pushes would not fit
                const unsigned need = (unsigned)__popc(sm);
                if (top - bot + need > cap) donate(top - bot + need - cap / 2u, true);
                const bool room = top - bot + need <= cap;
                if (!room && lane == 0) {
                    // ring and deque both full: these siblings are lost (flagged)
                    W.live_delta -= 3 * (long long)need;
                    atomicOr(A.status, ERR_QUEUE_FULL);
                }
                if (is_split) {
                    // children 1..3 wait on the deque; this lane continues with child 0
                    Entry e;
                    const RayId id = s_id[threadIdx.x];
                    e.key = make_key(id.pix << 2, id.level + 1, 1);
                    e.src = id.src;
                    e.r = R.r;
                    e.N = make_float4(R.N.x * 0.25f, NG > 1 ? R.N.y * 0.25f : 0.f,
                                      NG > 2 ? R.N.z * 0.25f : 0.f, NG > 3 ? R.N.w * 0.25f : 0.f);
                    if (room) stack[(top + __popc(sm & lt_mask)) & cmask] = e;
                    // children 1..3 carry exact FP32 quarters; child 0 (this lane)
                    // also inherits the parent's sub-ulp low part, so no photon
                    // is lost and no cell receives a spurious deposit
                    const float4 keep = R.Nl;
                    ev = start_ray<EXT>(A, e, 0, R);
                    fold_low(R.N.x, R.Nl.x, keep.x);
                    fold_low(R.N.y, R.Nl.y, keep.y);
                    fold_low(R.N.z, R.Nl.z, keep.z);
                    if (NG > 3) fold_low(R.N.w, R.Nl.w, keep.w);
                }
                {
                    const unsigned lv = __reduce_max_sync(FULL, is_split ? (unsigned)s_id[threadIdx.x].level : 0u);
                    if (lane == 0) W.maxlev = max(W.maxlev, lv);
                }
                __syncwarp();
                if (room) top += need;
            }
        }

        // ------------------------------------------------------ housekeeping
        round++;
        if ((round & (HEARTBEAT_EVERY - 1)) == 0) {
            flush_live();
            if (lane == 0) atomicAdd(A.heartbeat, 1u);
        }
        // share work with idle warps: give away the oldest pending subtrees
        if ((round & 15) == 0 && top - bot >= 2) {
            int want = 0;
            if (lane == 0) {
                const int idlew = ld_relaxed_i32(A.n_idle);
                if (idlew > 0) {
                    const unsigned long long qn = ld_relaxed(A.qtail) - ld_relaxed(A.qhead);
                    if (qn < (unsigned long long)idlew) want = 1;
                }
            }
            want = __shfl_sync(FULL, want, 0);
            if (want) donate(min(2u, top - bot - 1), false);
        }
    }

    // ------------------------------------------------------------ totals
    flush_live();
    // per-lane counts stay far below 2^32 per launch; warp sums are formed in
    // the 64-bit atomics below, lane by lane
    unsigned long long wseg = s_nseg[threadIdx.x];
    double rounding = s_round[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) {
        wseg += __shfl_down_sync(FULL, wseg, o);
        rounding += __shfl_down_sync(FULL, rounding, o);
    }
    __syncwarp();
    if (lane == 0) {
        atomicAdd(&A.counters[CNT_SEG], wseg);
        atomicAdd(&A.counters[CNT_SEG_TOTAL], wseg);
        atomicAdd(&A.counters[CNT_RAYS], W.nrays);
        atomicAdd(&A.counters[CNT_SPLIT], W.nsplit);
        atomicAdd(&A.counters[CNT_TERM], W.nterm);
        atomicAdd(&A.counters[CNT_ESC], W.nesc);
        atomicAdd(&A.counters[CNT_DONATE], W.ndon);
        atomicMax(&A.counters[CNT_MAXLEVEL], (unsigned long long)W.maxlev);
        if (W.esc != 0.0) atomicAdd(A.escaped, W.esc);
        if (rounding != 0.0) atomicAdd(A.rounding, rounding);
    }
}

// ------------------------------------------------------------------ prep
// absorber densities (Sec. 2.3) -> optical depth per cell length per group;
// zero the accumulators (Sec. 2.1 step i).  One thread per internal cell.
__global__ void k_prep(const PrepArgs P) {
    const uint64_t nbc = (uint64_t)P.nb * P.nb * P.nb * 512ull;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nbc;
         q += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t b = q >> 9;
        const uint32_t m = (uint32_t)(q & 511u);
        const int k = (int)((b % P.nb) * 8 + compact3(m));
        const int j = (int)(((b / P.nb) % P.nb) * 8 + compact3(m >> 1));
        const int i = (int)((b / ((uint64_t)P.nb * P.nb)) * 8 + compact3(m >> 2));
        float4 kap = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < P.n && j < P.n && k < P.n) {
            const uint64_t c = ((uint64_t)i * P.n + j) * P.n + k;
            const float nh = P.nH[c];
            const float n0 = nh * P.xHI[c];
            const float n1 = P.y * nh * P.xHeI[c];
            const float n2 = P.y * nh * P.xHeII[c];
            float kb[ARC_MAX_GROUPS];
#pragma unroll
            for (int g = 0; g < ARC_MAX_GROUPS; ++g)
                kb[g] = (g < P.ng) ? (P.sig_dx[0][g] * n0 + P.sig_dx[1][g] * n1 + P.sig_dx[2][g] * n2) : 0.f;
            kap = make_float4(kb[0], kb[1], kb[2], kb[3]);
        }
        P.rec[2 * q] = kap;
        P.rec[2 * q + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_validate(const float* nH, const float* xHI, const float* xHeI, const float* xHeII,
                           const float* T, long long ncell, unsigned int* status) {
    bool bad = false;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const float a = nH[c], b = xHI[c], d = xHeI[c], e = xHeII[c], t = T[c];
        const bool ok = isfinite(a) && isfinite(b) && isfinite(d) && isfinite(e) && isfinite(t) &&
                        a >= 0.f && b >= 0.f && b <= 1.f && d >= 0.f && d <= 1.f && e >= 0.f &&
                        e <= 1.f && d + e <= 1.0f + 1e-6f && t > 0.f;
        bad |= !ok;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, ERR_FIELDS);
}

__global__ void k_make_seeds(const SourceDev* src, int nsrc, int per_src, int l_base, Entry* seeds) {
    const long long total = (long long)nsrc * per_src;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(q / per_src), e = (int)(q % per_src);
        Entry it;
        it.key = make_key(4ull * (uint64_t)e, l_base, 0);
        it.src = (uint32_t)s;
        it.r = 0.0f;
        it.N = src[s].N0;
        seeds[q] = it;
    }
}

__global__ void k_reset(TraceArgs A, unsigned long long qcap, int nseeds) {
    for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < qcap;
         q += (unsigned long long)gridDim.x * blockDim.x)
        A.qseq[q] = q;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *A.qhead = 0;
        *A.qtail = 0;
        *A.seed_head = 0;
        *A.live = 4ll * nseeds;
        *A.n_idle = 0;
        *A.heartbeat = 0;
        *A.escaped = 0.0;
        *A.rounding = 0.0;
        if (A.thin) *A.thin = 0.0;
        for (int i = 0; i < CNT_N; ++i) A.counters[i] = 0;
        A.counters[CNT_TRACES_TOTAL] += 1;
        if (A.nrec) *A.nrec = 0;
        atomicAnd(A.status, ~(ERR_TIMEOUT | ERR_QUEUE_FULL | ERR_RECORDS | ERR_CAS_SPIN));
    }
}

// ------------------------------------------------------------------ finalize
// Per cell: D_b photons absorbed in group b (FP32 sum).  Eq. (ion)
// splits D_b over the absorbers in proportion to sigma_{s,b} n_s and divides
// by V n_s; with kappa_b = sum_s sigma_{s,b} n_s this is
//   Gamma_s = (PHOT_UNIT / V) sum_b D_b sigma_{s,b} / kappa_b,
// and the heating per absorber adds the excess energy E_b - E_s (Sec. 2.8).
__global__ void k_finalize(const FinalizeArgs F) {
    const uint64_t n3 = (uint64_t)F.n * F.n * F.n;
    double part = 0.0;
    for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n3;
         c += (uint64_t)gridDim.x * blockDim.x) {
        const int k = (int)(c % F.n);
        const int j = (int)((c / F.n) % F.n);
        const int i = (int)(c / ((uint64_t)F.n * F.n));
        const uint64_t q = brick_index(i, j, k, F.nb);
        const float4 a = F.rec[2 * q + 1];
        part += ((double)a.x + (double)a.y) + ((double)a.z + (double)a.w);
        const float D[4] = {a.x, a.y, a.z, a.w};
        const float nh = F.nH[c];
        const float ns[3] = {nh * F.xHI[c], F.y * nh * F.xHeI[c], F.y * nh * F.xHeII[c]};
        float g[3] = {0.f, 0.f, 0.f}, h[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int b = 0; b < ARC_MAX_GROUPS; ++b) {
            if (b >= F.ng || D[b] == 0.f) continue;
            const float kb = F.sig[0][b] * ns[0] + F.sig[1][b] * ns[1] + F.sig[2][b] * ns[2];
            if (!(kb > 0.f)) continue;   // no absorber of this group in the cell
            const float w = D[b] * F.scale;
#pragma unroll
            for (int s = 0; s < 3; ++s) {
                const float rate = w * (F.sig[s][b] / kb);
                g[s] += rate;
                h[s] += rate * F.egap_erg[s][b];
            }
        }
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            F.gamma[s * n3 + c] = g[s];
            F.heat[s * n3 + c] = h[s];
        }
    }
    // block partial of the absorbed photons
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(FULL, part, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        F.absorbed_part[blockIdx.x] = t;
    }
}

__global__ void k_budget(const double* part, int nparts, const double* escaped, const double* rounding,
                         const double* thin, double* out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(FULL, s, o);
    __shared__ double ws[32];
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
        // the cell sums plus what their FP32 additions rounded away, less the
        // thin fill's photons, which no ray carried (Sec. 2.6)
        out[0] = t + *rounding - (thin ? *thin : 0.0);
        out[1] = *escaped;
    }
}

// ------------------------------------------------------------------ thin region
// Sec. 2.6.  begin: the emitted rays of each source start at its radius R, and
// the radius candidates are reset to +inf.
__global__ void k_thin_begin(Entry* seeds, int nseeds, const float* rthin, float* rnext, int nsrc) {
    const int stride = gridDim.x * blockDim.x;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nseeds; q += stride)
        seeds[q].r = rthin[seeds[q].src];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsrc; s += stride) rnext[s] = INFINITY;
}

// Cells whose centre lies within R of a source absorb, per group, the thin
// limit of Eq. (ion) summed over the rays crossing them: S_b kappa_b V /
// (4 pi r^2) (kappa_b per cell length, r in cells from the source to the
// centre, floored at half a cell where 1/r^2 diverges).  The photons go through
// the same returning atomics and rounding ledger as the rays' deposits and are
// counted in the thin ledger, so that the budget still closes over the rays.
// Grid: x strides over the cube of cells around one source, y over sources.
__global__ void k_thin_fill(const ThinFillArgs F) {
    constexpr float INV_4PI = 0.0795774715459476679f;
    double got = 0.0, err = 0.0;
    for (int s = blockIdx.y; s < F.nsrc; s += gridDim.y) {
        const float R = F.rthin[s];
        if (!(R > 0.0f)) continue;
        const float4 pt = F.src[s].pos_thr;
        const float4 N0 = F.src[s].N0;
        const float4 S = make_float4(N0.x * F.nbase, N0.y * F.nbase, N0.z * F.nbase, N0.w * F.nbase);
        // cells with centre c + 1/2 in [o - R, o + R] per axis, clipped to the
        // box (the extent is capped at 2n so that the bounds stay integers)
        const float o[3] = {pt.x, pt.y, pt.z};
        const float Rb = fminf(R, 2.0f * (float)F.n);
        int lo[3], m[3];
        bool empty = false;
        for (int a = 0; a < 3; ++a) {
            lo[a] = max(0, (int)ceilf(o[a] - Rb - 0.5f));
            const int hi = min(F.n - 1, (int)floorf(o[a] + Rb - 0.5f));
            m[a] = hi - lo[a] + 1;
            empty |= m[a] <= 0;
        }
        if (empty) continue;
        const long long myz = (long long)m[1] * m[2];
        const long long tot = (long long)m[0] * myz;
        const float R2 = R * R;
        for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < tot;
             q += (long long)gridDim.x * blockDim.x) {
            const int i = lo[0] + (int)(q / myz);
            const long long rem = q % myz;
            const int j = lo[1] + (int)(rem / m[2]);
            const int k = lo[2] + (int)(rem % m[2]);
            const float dx = (float)i + 0.5f - o[0], dy = (float)j + 0.5f - o[1], dz = (float)k + 0.5f - o[2];
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (!(r2 < R2)) continue;
            const float f = INV_4PI / fmaxf(r2, 0.25f);
            const uint64_t idx = brick_index(i, j, k, F.nb);
            const float4 kap = F.rec[2 * idx];
            const float4 D = make_float4(S.x * kap.x * f, S.y * kap.y * f, S.z * kap.z * f, S.w * kap.w * f);
            if (D.x == 0.f && D.y == 0.f && D.z == 0.f && D.w == 0.f) continue;
            err += (double)deposit<4>(F.rec, idx, D, make_float4(0.f, 0.f, 0.f, 0.f));
            got += ((double)D.x + (double)D.y) + ((double)D.z + (double)D.w);
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        got += __shfl_down_sync(FULL, got, o);
        err += __shfl_down_sync(FULL, err, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (got != 0.0) atomicAdd(F.thin, got);
        if (err != 0.0) atomicAdd(F.rounding, err);
    }
}

// commit: the radius each source measured becomes the one of the next trace
// (0 when no ray of the source offered one)
__global__ void k_thin_commit(float* rthin, const float* rnext, int nsrc) {
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < nsrc; s += gridDim.x * blockDim.x) {
        const float v = rnext[s];
        rthin[s] = (v < INFINITY) ? v : 0.0f;
    }
}

}  // namespace

// ------------------------------------------------------------------ launchers
int trace_smem_bytes(int block, int stack_log2) {
    return (block / 32) * (1 << stack_log2) * (int)sizeof(Entry);
}
// the tracer is specialised on the number of frequency groups carried, on the
// per-ray records (test aid) and on the extended emission (masks, Sec. 2.2;
// optically thin radius, Sec. 2.6)
template <bool REC, bool EXT>
const void* trace_kernel_ng(int ng) {
    if (ng <= 1) return (const void*)k_trace<1, REC, EXT>;
    if (ng <= 3) return (const void*)k_trace<3, REC, EXT>;
    return (const void*)k_trace<4, REC, EXT>;
}
const void* trace_kernel_ptr(int ng, bool rec, bool ext) {
    if (rec) return ext ? trace_kernel_ng<true, true>(ng) : trace_kernel_ng<true, false>(ng);
    return ext ? trace_kernel_ng<false, true>(ng) : trace_kernel_ng<false, false>(ng);
}

cudaError_t launch_prep(const PrepArgs& a, cudaStream_t s) {
    k_prep<<<152 * 8, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_validate(const float* nH, const float* xHI, const float* xHeI,
                            const float* xHeII, const float* T, long long ncell,
                            unsigned int* status, cudaStream_t s) {
    k_validate<<<152 * 4, 256, 0, s>>>(nH, xHI, xHeI, xHeII, T, ncell, status);
    return cudaGetLastError();
}
cudaError_t launch_make_seeds(const SourceDev* src, int nsrc, int l_base, Entry* seeds,
                              cudaStream_t s) {
    const int per_src = 3 << (2 * l_base);
    const long long total = (long long)nsrc * per_src;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_make_seeds<<<blocks, 256, 0, s>>>(src, nsrc, per_src, l_base, seeds);
    return cudaGetLastError();
}
cudaError_t launch_seed_reset(const TraceArgs& a, unsigned long long qcap, int nseeds, cudaStream_t s) {
    k_reset<<<152 * 2, 256, 0, s>>>(a, qcap, nseeds);
    return cudaGetLastError();
}
template <bool REC, bool EXT>
void launch_trace_ng(const TraceArgs& a, int grid, int block, int smem, cudaStream_t s) {
    if (a.ng <= 1) k_trace<1, REC, EXT><<<grid, block, smem, s>>>(a);
    else if (a.ng <= 3) k_trace<3, REC, EXT><<<grid, block, smem, s>>>(a);
    else k_trace<4, REC, EXT><<<grid, block, smem, s>>>(a);
}
void fill_sincos_table(TraceArgs& a) {
    for (int j = -16; j <= 16; ++j) {
        const double x = M_PI * (double)j / 64.0;
        const double sd = sin(x), cd = cos(x);
        const float sh = (float)sd, ch = (float)cd;
        a.sincos[j + 16] = make_float4(sh, (float)(sd - (double)sh), ch, (float)(cd - (double)ch));
    }
}

cudaError_t launch_trace(const TraceArgs& a, int grid, int block, cudaStream_t s) {
    const int smem = trace_smem_bytes(block, a.stack_log2);
    const bool ext = a.rnext != nullptr || a.open != nullptr;
    if (a.recs != nullptr) {   // test aid: per-ray records (cell-visit counts)
        if (ext) launch_trace_ng<true, true>(a, grid, block, smem, s);
        else launch_trace_ng<true, false>(a, grid, block, smem, s);
    } else {
        if (ext) launch_trace_ng<false, true>(a, grid, block, smem, s);
        else launch_trace_ng<false, false>(a, grid, block, smem, s);
    }
    return cudaGetLastError();
}
cudaError_t launch_thin_begin(Entry* seeds, int nseeds, const float* rthin, float* rnext, int nsrc,
                              cudaStream_t s) {
    const int work = max(nseeds, nsrc);
    int blocks = (work + 255) / 256;
    blocks = max(1, min(blocks, 152 * 4));
    k_thin_begin<<<blocks, 256, 0, s>>>(seeds, nseeds, rthin, rnext, nsrc);
    return cudaGetLastError();
}
cudaError_t launch_thin_fill(const ThinFillArgs& a, cudaStream_t s) {
    if (a.nsrc <= 0) return cudaSuccess;
    const dim3 grid(16, (unsigned)min(a.nsrc, 65535));
    k_thin_fill<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_thin_commit(float* rthin, const float* rnext, int nsrc, cudaStream_t s) {
    if (nsrc <= 0) return cudaSuccess;
    k_thin_commit<<<(nsrc + 255) / 256, 256, 0, s>>>(rthin, rnext, nsrc);
    return cudaGetLastError();
}
cudaError_t launch_finalize(const FinalizeArgs& a, int blocks, cudaStream_t s) {
    k_finalize<<<blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_budget(const double* part, int nparts, const double* escaped, const double* rounding,
                          const double* thin, double* out, cudaStream_t s) {
    k_budget<<<1, 256, 0, s>>>(part, nparts, escaped, rounding, thin, out);
    return cudaGetLastError();
}

}  // namespace arc
