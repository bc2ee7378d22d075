// arc_chem.cu -- per-cell H/He ionisation and energy update of libarc (sm_103a).
//
// Sec. 2.7 (Eq. diffeq in the D - C n form of Eq. anninos, backward
// difference, sub-cycled between radiative-transfer steps with the step
// limited to a fraction eps of the change of E, n_HI, n_HII, n_HeI, n_HeII
// and n_HeIII: every quantity the equations track) and Sec. 2.8
// (photoheating minus cooling).  One thread per cell.
//
// The update is written per hydrogen atom: abundances a_s = n_s / n_H and
// energy e = E / n_H.  This is the density form divided by n_H; it keeps the
// FP32 cooling terms of low-density cells (n_e n_s ~ 1e-10) far from the FP32
// underflow that the volumetric form would reach.  Sub-steps of cells whose
// neutral fraction is below x_fp64 do the species update in FP64.
//
// Rate fits: Hui & Gnedin (1997) case-B recombination, collisional
// ionisation and recombination cooling; Cen (1992) collisional excitation,
// dielectronic recombination and the free-free Gaunt factor; Compton cooling
// off the CMB.  Evaluated in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "arc_internal.cuh"

namespace arc {

namespace {

constexpr int MAX_SUBSTEPS = 100000;
constexpr float T_FLOOR = 1.0f;
constexpr float TH_HI = 157807.0f, TH_HEI = 285335.0f, TH_HEII = 631515.0f;
constexpr float KB = 1.380649e-16f;

struct Coef {
    float aH, a2, a3;     // recombination HII, HeII (+ dielectronic), HeIII [cm^3/s]
    float b0, b1, b2;     // collisional ionisation HI, HeI, HeII [cm^3/s]
};

// Transcendentals of the rate fits.  The plain solver evaluates them with
// the accurate library functions; the surrogate's predictor and residual
// check use the fast hardware forms, whose ~1e-6 relative error is far below
// the check's tolerances.
struct ExactMath {
    static __device__ __forceinline__ float pow(float x, float e) { return powf(x, e); }
    static __device__ __forceinline__ float exp(float x) { return expf(x); }
    static __device__ __forceinline__ float lg10(float x) { return log10f(x); }
};
struct FastMath {
    static __device__ __forceinline__ float pow(float x, float e) { return __powf(x, e); }
    static __device__ __forceinline__ float exp(float x) { return __expf(x); }
    static __device__ __forceinline__ float lg10(float x) { return __log10f(x); }
};

template <class M>
__device__ __forceinline__ float hg_alpha(float lam) {
    return 2.753e-14f * M::pow(lam, 1.5f) / M::pow(1.0f + M::pow(lam * (1.0f / 2.740f), 0.407f), 2.242f);
}
template <class M>
__device__ __forceinline__ float hg_recool(float T, float lam) {
    return 3.435e-30f * T * M::pow(lam, 1.970f) / M::pow(1.0f + M::pow(lam * (1.0f / 2.250f), 0.376f), 3.720f);
}
template <class M>
__device__ __forceinline__ float dielectronic_shape(float T) {
    return M::pow(T, -1.5f) * M::exp(-4.7e5f / T) * (1.0f + 0.3f * M::exp(-9.4e4f / T));
}

template <class M = ExactMath>
__device__ __forceinline__ Coef coefficients(float T, const ChemArgs& C) {
    const float lHI = 2.0f * TH_HI / T, lHeI = 2.0f * TH_HEI / T, lHeII = 2.0f * TH_HEII / T;
    Coef r;
    r.aH = C.alpha_fixed > 0.0f ? C.alpha_fixed : hg_alpha<M>(lHI);
    r.a2 = 1.26e-14f * M::pow(lHeI, 0.750f) + 1.90e-3f * dielectronic_shape<M>(T);
    r.a3 = 2.0f * hg_alpha<M>(lHeII);
    if (C.coll_ion) {
        const float t32 = M::pow(T, -1.5f);
        r.b0 = 21.11f * t32 * M::exp(-0.5f * lHI) * M::pow(lHI, -1.089f) /
               M::pow(1.0f + M::pow(lHI * (1.0f / 0.354f), 0.874f), 1.101f);
        r.b1 = 32.38f * t32 * M::exp(-0.5f * lHeI) * M::pow(lHeI, -1.146f) /
               M::pow(1.0f + M::pow(lHeI * (1.0f / 0.416f), 0.987f), 1.056f);
        r.b2 = 19.95f * t32 * M::exp(-0.5f * lHeII) * M::pow(lHeII, -1.089f) /
               M::pow(1.0f + M::pow(lHeII * (1.0f / 0.553f), 0.735f), 1.275f);
    } else {
        r.b0 = r.b1 = r.b2 = 0.0f;
    }
    return r;
}

// Cooling per hydrogen atom [erg/s]: Lambda / n_H for abundances a0 = HI,
// a1 = HeI, a2 = HeII per H and electrons xe per H.
template <class M = ExactMath>
__device__ __forceinline__ float cooling_per_h(float T, float nH, float a0, float a1, float a2,
                                               float xe, const Coef& r, const ChemArgs& C) {
    const float lHI = 2.0f * TH_HI / T, lHeI = 2.0f * TH_HEI / T, lHeII = 2.0f * TH_HEII / T;
    const float aHII = 1.0f - a0;
    const float a3 = fmaxf(C.y - a1 - a2, 0.0f);          // HeIII per H
    const float nxe = nH * xe;                             // n_e [cm^-3]
    float L = r.b0 * a0 * (KB * TH_HI) + r.b1 * a1 * (KB * TH_HEI) + r.b2 * a2 * (KB * TH_HEII);
    // HeIII recombination is hydrogenic (Z = 2): Z^3 times the HII cooling at
    // T / Z^2, i.e. the fit at lHeII with its temperature prefactor scaled
    L += hg_recool<M>(T, lHI) * aHII + 1.26e-14f * M::pow(lHeI, 0.750f) * KB * T * a2 +
         8.0f * hg_recool<M>(T * (TH_HI / TH_HEII), lHeII) * a3 + 1.24e-13f * dielectronic_shape<M>(T) * a2;
    const float sq = 1.0f + sqrtf(T * 1e-5f);
    L += 7.5e-19f * M::exp(-118348.0f / T) / sq * a0 + 5.54e-17f * M::pow(T, -0.397f) * M::exp(-473638.0f / T) / sq * a2;
    const float lg = M::lg10(T) - 5.5f;
    const float gff = 1.1f + 0.34f * M::exp(-lg * lg * (1.0f / 3.0f));
    L += 1.42e-27f * gff * sqrtf(T) * (aHII + a2 + 4.0f * a3);
    L *= nxe;
    if (C.compton) L += C.compton_coef * (T - C.tcmb) * xe;
    return L;
}

template <typename R>
__device__ __forceinline__ void species_update(R h, R nH, R y, R G0, R G1, R G2, const Coef& c,
                                               R xe, R& a0, R& a1, R& a2) {
    const R nxe = nH * xe;
    // HI:  da0/dt = alpha n_e (1 - a0) ... written D - C a0 with D = alpha n_e
    const R DH = (R)c.aH * nxe;
    const R CH = G0 + ((R)c.b0 + (R)c.aH) * nxe;
    a0 = (a0 + h * DH) / ((R)1 + h * CH);
    // HeI: source recombination of HeII, sink photo + collisional ionisation
    const R C1 = G1 + (R)c.b1 * nxe;
    const R D1 = (R)c.a2 * nxe * a2;
    a1 = (a1 + h * D1) / ((R)1 + h * C1);
    if (a1 > y) a1 = y;
    // HeII: sources ionisation of HeI and recombination of HeIII (= y - a1 - a2)
    const R C2 = G2 + ((R)c.b2 + (R)c.a2 + (R)c.a3) * nxe;
    const R D2 = (G1 + (R)c.b1 * nxe) * a1 + (R)c.a3 * nxe * (y - a1);
    a2 = (a2 + h * D2) / ((R)1 + h * C2);
    if (a2 > y - a1) a2 = y - a1;
    if (a2 < (R)0) a2 = (R)0;
}

__global__ void __launch_bounds__(256) k_chem(const ChemArgs C) {
    unsigned long long nsub_tot = 0, nsub64 = 0, capped = 0;
    const float y = C.y;
    const long long count = C.list ? (long long)*C.list_count : C.ncell;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const long long c = C.list ? (long long)C.list[i] : i;
        const float nH = C.nH[c];
        if (!(nH > 0.0f)) continue;
        float a0 = C.xHI[c], a1 = y * C.xHeI[c], a2 = y * C.xHeII[c], T = C.T[c];
        const float G0 = C.gamma[c], G1 = C.gamma[C.ncell + c], G2 = C.gamma[2 * C.ncell + c];
        const float H0 = C.heat[c], H1 = C.heat[C.ncell + c], H2 = C.heat[2 * C.ncell + c];
        const float dt = (float)C.dt;
        // elapsed time as an unevaluated pair (t_hi + t_lo): sub-steps can be
        // far below one ulp of dt, so a plain FP32 sum would stall
        float t_hi = 0.0f, t_lo = 0.0f;
        int nsub = 0;
        bool cap = false;
        for (;;) {
            if (nsub >= MAX_SUBSTEPS) {
                cap = true;
                break;
            }
            const float xe = (1.0f - a0) + a2 + 2.0f * (y - a1 - a2);
            const Coef r = coefficients(T, C);
            const float nxe = nH * xe;
            const float dHI = r.aH * nxe * (1.0f - a0) - (G0 + r.b0 * nxe) * a0;
            float h = __fsub_rn(__fsub_rn(dt, t_hi), t_lo);
            bool last = true;
            const float lim = C.eps * fmaxf(fminf(a0, 1.0f - a0), C.xfloor);
            if (fabsf(dHI) * h > lim) {
                h = lim / fabsf(dHI);
                last = false;
            }
            // ... and of HeI, HeII, HeIII (each floored at xfloor of the helium):
            // the limit covers every quantity the equations track (Sec. 2.7)
            if (y > 0.0f) {
                const float a3 = y - a1 - a2;
                const float d1 = r.a2 * nxe * a2 - (G1 + r.b1 * nxe) * a1;
                const float d3 = (G2 + r.b2 * nxe) * a2 - r.a3 * nxe * a3;
                const float dh[3] = {d1, -d1 - d3, d3};
                const float ah[3] = {a1, a2, a3};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float limk = C.eps * fmaxf(ah[k], C.xfloor * y);
                    if (fabsf(dh[k]) * h > limk) {
                        h = limk / fabsf(dh[k]);
                        last = false;
                    }
                }
            }
            float e = 0.0f, edot = 0.0f;
            if (!C.isothermal) {
                e = 1.5f * KB * T * (1.0f + y + xe);
                edot = (a0 * H0 + a1 * H1 + a2 * H2) - cooling_per_h(T, nH, a0, a1, a2, xe, r, C);
                if (fabsf(edot) * h > C.eps * e) {
                    h = C.eps * e / fabsf(edot);
                    last = false;
                }
            }
            if (a0 < C.xfloor) {
                double d0 = a0, d1 = a1, d2 = a2;
                species_update<double>((double)h, (double)nH, (double)y, (double)G0, (double)G1,
                                       (double)G2, r, (double)xe, d0, d1, d2);
                a0 = (float)d0;
                a1 = (float)d1;
                a2 = (float)d2;
                nsub64++;
            } else {
                species_update<float>(h, nH, y, G0, G1, G2, r, xe, a0, a1, a2);
            }
            if (!C.isothermal) {
                const float xe1 = (1.0f - a0) + a2 + 2.0f * (y - a1 - a2);
                T = fmaxf((e + h * edot) / (1.5f * KB * (1.0f + y + xe1)), T_FLOOR);
            }
            nsub++;
            if (last) break;
            const float s = __fadd_rn(t_hi, h);
            const float bb = __fsub_rn(s, t_hi);
            t_lo = __fadd_rn(t_lo, __fadd_rn(__fsub_rn(t_hi, __fsub_rn(s, bb)), __fsub_rn(h, bb)));
            t_hi = s;
        }
        nsub_tot += (unsigned long long)nsub;
        capped += cap ? 1ull : 0ull;
        C.xHI[c] = a0;
        if (y > 0.0f) {
            C.xHeI[c] = a1 / y;
            C.xHeII[c] = a2 / y;
        }
        C.T[c] = T;
    }
    for (int o = 16; o > 0; o >>= 1) {
        nsub_tot += __shfl_down_sync(0xFFFFFFFFu, nsub_tot, o);
        nsub64 += __shfl_down_sync(0xFFFFFFFFu, nsub64, o);
        capped += __shfl_down_sync(0xFFFFFFFFu, capped, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nsub_tot) atomicAdd(&C.counters[0], nsub_tot);
        if (nsub64) atomicAdd(&C.counters[1], nsub64);
        if (capped) {
            atomicAdd(&C.counters[2], capped);
            atomicOr(C.status, ERR_SUBSTEP);
        }
    }
}

// ------------------------------------------------------------------ surrogate
// Tensor-core MLP (mma.sync m16n8k16, BF16 in, FP32 accumulate) over tiles of
// 16 cells per warp.  The activations stay in registers between layers: the
// FP32 accumulator fragment of two adjacent 8-column output tiles is, after
// bias and SiLU, exactly the BF16 A fragment of the next layer's 16-wide
// input tile.
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}
// SiLU for the inference tiles: the fast exponential and a correctly rounded
// reciprocal keep its relative error near 1e-7, far below the BF16 rounding
// (2^-9) that every activation takes next
__device__ __forceinline__ float silu(float z) { return z * __frcp_rn(1.0f + __expf(-z)); }

// out = SiLU(in W^T + b) for a 16-row tile; in has KT 16-wide k-tiles, out 64 columns
template <int KT>
__device__ __forceinline__ void dense_silu(const uint32_t (&ain)[KT][4], uint32_t (&aout)[4][4],
                                           const unsigned short* W, int ldw, const float* bias, int g, int t4) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int kt = 0; kt < KT; ++kt) {
            const unsigned short* wr = W + (8 * j + g) * ldw + 16 * kt + 2 * t4;
            mma_bf16(c, ain[kt], *reinterpret_cast<const uint32_t*>(wr), *reinterpret_cast<const uint32_t*>(wr + 8));
        }
        const float b0 = bias[8 * j + 2 * t4], b1 = bias[8 * j + 2 * t4 + 1];
        const uint32_t top = pack_bf16(silu(c[0] + b0), silu(c[1] + b1));
        const uint32_t bot = pack_bf16(silu(c[2] + b0), silu(c[3] + b1));
        if ((j & 1) == 0) {
            aout[j >> 1][0] = top;
            aout[j >> 1][1] = bot;
        } else {
            aout[j >> 1][2] = top;
            aout[j >> 1][3] = bot;
        }
    }
}

// The rate equations of Eq. (anninos) are linear in the abundances once n_e
// and T are fixed.  With the coefficients frozen (evaluated at abundances
// c0..c2 per H and temperature Tc) they integrate exactly over dt:
//   HI:  a0' = D - C a0,
//   He:  v' = A v + c for v = (HeI, HeII) per H, HeIII = y - HeI - HeII,
//        whose matrix has real eigenvalues lam1 >= lam2 (the three-state
//        chain is a birth-death process, similar to a symmetric matrix),
// both written v(dt) = v0 + phi(A) (A v0 + c), phi(A) = int_0^dt e^{A t} dt,
// which stays finite as the rates vanish.

// phi1(u) = (e^u - 1) / u and phi2(u) = (e^u - 1 - u) / u^2 (the integral of
// phi1(u s) s over s in [0, 1]) with their derivatives, for u <= 0: series
// for |u| < 0.1, where the closed forms cancel; beyond, the closed forms with
// the fast exponential keep a relative error below ~1e-4 (surrogate use only)
__device__ __forceinline__ float phi1(float u) {
    if (fabsf(u) < 0.1f) return 1.0f + u * (0.5f + u * (1.0f / 6.0f + u * (1.0f / 24.0f + u * (1.0f / 120.0f))));
    return __fdividef(__expf(u) - 1.0f, u);
}
__device__ __forceinline__ float phi1_d(float u) {
    if (fabsf(u) < 0.1f) return 0.5f + u * (1.0f / 3.0f + u * (0.125f + u * (1.0f / 30.0f + u * (1.0f / 144.0f))));
    const float e = __expf(u);
    return __fdividef(u * e - (e - 1.0f), u * u);
}
__device__ __forceinline__ float phi2(float u) {
    if (fabsf(u) < 0.1f) return 0.5f + u * (1.0f / 6.0f + u * (1.0f / 24.0f + u * (1.0f / 120.0f)));
    return __fdividef(__expf(u) - 1.0f - u, u * u);
}
__device__ __forceinline__ float phi2_d(float u) {
    if (fabsf(u) < 0.1f) return 1.0f / 6.0f + u * (1.0f / 12.0f + u * (1.0f / 40.0f + u * (1.0f / 180.0f)));
    return __fdividef(phi1(u) - 2.0f * phi2(u), u);
}
// divided difference f[u1, u2] for u1 >= u2, by the derivative at the midpoint
// where the two are close
template <float (*F)(float), float (*FD)(float)>
__device__ __forceinline__ float divdiff(float u1, float u2) {
    const float du = u1 - u2, um = 0.5f * (u1 + u2);
    return du > 1e-2f * fmaxf(1.0f, fabsf(um)) ? (F(u1) - F(u2)) / du : FD(um);
}

// Frozen-coefficient solution over dt from (a0, a1, a2) with coefficients
// evaluated at abundances (c0, c1, c2) and rates r; with ints != nullptr
// also the time integrals int_0^dt a_s dt (for the photoheating).
// Matrix functions of the 2x2 He system use f(A dt) = f(u2) I +
// f[u1, u2] dt (A - lam2 I), u = lam dt.
__device__ void frozen_abundances(float nH, float y, float c0, float c1, float c2, const Coef& r,
                                  const float (&G)[3], float a0, float a1, float a2, float dt, float& e0,
                                  float& e1, float& e2, float* ints = nullptr) {
    const float ne = nH * ((1.0f - c0) + c2 + 2.0f * (y - c1 - c2));
    const float CH = G[0] + (r.b0 + r.aH) * ne, DH = r.aH * ne;
    const float fH = DH - CH * a0;
    e0 = a0 + dt * phi1(-CH * dt) * fH;
    e1 = a1;
    e2 = a2;
    if (ints) {
        ints[0] = dt * a0 + dt * dt * phi2(-CH * dt) * fH;
        ints[1] = dt * a1;
        ints[2] = dt * a2;
    }
    if (!(y > 0.0f)) return;
    // helium chain: A = [[-k1, r2], [k1 - r3, -(k2 + r2 + r3)]], c = (0, r3 y)
    const float k1 = G[1] + r.b1 * ne, k2 = G[2] + r.b2 * ne, r2 = r.a2 * ne, r3 = r.a3 * ne;
    const float A11 = -k1, A12 = r2, A21 = k1 - r3, A22 = -(k2 + r2 + r3);
    const float tr = A11 + A22;
    const float det = k1 * (k2 + r3) + r2 * r3;   // = A11 A22 - A12 A21, all terms >= 0
    const float hd = 0.5f * (A11 - A22);
    const float mu = sqrtf(fmaxf(hd * hd + A12 * A21, 0.0f));
    const float l2 = 0.5f * tr - mu;               // most negative eigenvalue
    const float l1 = l2 < 0.0f ? fminf(det / l2, 0.0f) : 0.0f;
    const float u1 = l1 * dt, u2 = l2 * dt;
    const float f1 = A11 * a1 + A12 * a2, f2 = A21 * a1 + A22 * a2 + r3 * y;   // v' at the start
    const float m1 = (A11 - l2) * f1 + A12 * f2, m2 = A21 * f1 + (A22 - l2) * f2;   // (A - lam2 I) f
    // v(dt) = v0 + dt phi1(A dt) f
    const float q0 = dt * phi1(u2), q1 = dt * dt * divdiff<phi1, phi1_d>(u1, u2);
    e1 = fminf(fmaxf(a1 + q0 * f1 + q1 * m1, 0.0f), y);
    e2 = fminf(fmaxf(a2 + q0 * f2 + q1 * m2, 0.0f), y - e1);
    if (ints) {
        // int v dt = dt v0 + dt^2 phi2(A dt) f
        const float w0 = dt * dt * phi2(u2), w1 = dt * dt * dt * divdiff<phi2, phi2_d>(u1, u2);
        ints[1] = dt * a1 + w0 * f1 + w1 * m1;
        ints[2] = dt * a2 + w0 * f2 + w1 * m2;
    }
}

// Physics predictor of a step, which the network corrects: abundances from
// the rate equations frozen at the start state; energy from the photoheating
// of those abundance histories minus the cooling of the start state.
__device__ void surrogate_predictor(float nH, float y, float a0, float a1, float a2, float T, const float (&G)[3],
                                    const float (&H)[3], float dt, const ChemArgs& C, float& p0, float& p1,
                                    float& p2, float& pT) {
    const Coef r = coefficients<FastMath>(T, C);
    float I[3];
    frozen_abundances(nH, y, a0, a1, a2, r, G, a0, a1, a2, dt, p0, p1, p2, I);
    pT = T;
    if (!C.isothermal) {
        const float xe0 = (1.0f - a0) + a2 + 2.0f * (y - a1 - a2);
        const float xe1 = (1.0f - p0) + p2 + 2.0f * (y - p1 - p2);
        const float E0 = 1.5f * KB * T * (1.0f + y + xe0);
        const float E1 = E0 + (I[0] * H[0] + I[1] * H[1] + I[2] * H[2]) -
                         dt * cooling_per_h<FastMath>(T, nH, a0, a1, a2, xe0, r, C);
        pT = fmaxf(E1 / (1.5f * KB * (1.0f + y + xe1)), T_FLOOR);
    }
}

// Residual check of a surrogate step (start a0..a2 per H and T; prediction
// s0..s2, sT).  The step is re-integrated in two halves, each with the
// frozen-coefficient solution whose coefficients are taken on the straight
// path from start to prediction at 1/4 and 3/4 of the step (a second-order
// integrator whose coefficients come from the prediction itself).  Every
// predicted abundance must agree with it within tol_x (He per He atom), and
// the predicted energy with E0 plus the photoheating of its abundance
// histories minus the cooling at the two points, within tol_e of the energy.
// One half-step evaluation (the midpoint alone) is fooled where the
// coefficients vary strongly along the step, e.g. an ionisation front
// crossing the cell; two are not, on the cosmic-field states tested.
__device__ bool surrogate_accept(float nH, float y, float a0, float a1, float a2, float T, float s0, float s1,
                                 float s2, float sT, const float (&G)[3], const float (&H)[3], float dt,
                                 const ChemArgs& C, float tol_x, float tol_e) {
    float e0 = a0, e1 = a1, e2 = a2;
    float dE = 0.0f;
    const float h = 0.5f * dt;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const float f = j ? 0.75f : 0.25f;
        const float m0 = a0 + f * (s0 - a0), m1 = a1 + f * (s1 - a1), m2 = a2 + f * (s2 - a2);
        const float Tm = T + f * (sT - T);
        const Coef r = coefficients<FastMath>(Tm, C);
        float I[3];
        frozen_abundances(nH, y, m0, m1, m2, r, G, e0, e1, e2, h, e0, e1, e2, I);
        if (!C.isothermal) {
            const float xe = (1.0f - m0) + m2 + 2.0f * (y - m1 - m2);
            dE += (I[0] * H[0] + I[1] * H[1] + I[2] * H[2]) - h * cooling_per_h<FastMath>(Tm, nH, m0, m1, m2, xe, r, C);
        }
    }
    const float th = tol_x * y;
    if (!(fabsf(e0 - s0) <= tol_x) || !(fabsf(e1 - s1) <= th) || !(fabsf(e2 - s2) <= th)) return false;
    if (!C.isothermal) {
        const float xe0 = (1.0f - a0) + a2 + 2.0f * (y - a1 - a2);
        const float xe1 = (1.0f - s0) + s2 + 2.0f * (y - s1 - s2);
        const float E0 = 1.5f * KB * T * (1.0f + y + xe0), E1 = 1.5f * KB * sT * (1.0f + y + xe1);
        if (!(fabsf(E1 - E0 - dE) <= tol_e * fmaxf(E0, E1))) return false;
    }
    return true;
}

// Normalised features of one cell -> one row of the feature tile as BF16
// hi (columns 0..15) and lo (columns 16..31) halves.
__device__ __forceinline__ void store_features(unsigned short* row, const float (&f)[MLP_IN], const MlpDev& w) {
#pragma unroll
    for (int k = 0; k < 16; k += 2) {
        const float v0 = k < MLP_IN ? (f[k] - w.in_mu[k]) / w.in_sd[k] : 0.f;
        const float v1 = k + 1 < MLP_IN ? (f[k + 1] - w.in_mu[k + 1]) / w.in_sd[k + 1] : 0.f;
        const __nv_bfloat162 hi = __floats2bfloat162_rn(v0, v1);
        const float2 hf = __bfloat1622float2(hi);
        *reinterpret_cast<__nv_bfloat162*>(row + k) = hi;
        *reinterpret_cast<__nv_bfloat162*>(row + 16 + k) = __floats2bfloat162_rn(v0 - hf.x, v1 - hf.y);
    }
}

// The network on one 16-cell tile: normalised BF16 features ft[16][MLP_LD1]
// (shared memory) -> normalised outputs out[16][4] (shared memory).
__device__ __forceinline__ void mlp_tile(const unsigned short* ft, const MlpDev& w, float (*out)[4], int g, int t4) {
    uint32_t ain[2][4];
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {   // hi and lo halves of the inputs
        ain[kt][0] = *reinterpret_cast<const uint32_t*>(ft + g * MLP_LD1 + 16 * kt + 2 * t4);
        ain[kt][1] = *reinterpret_cast<const uint32_t*>(ft + (g + 8) * MLP_LD1 + 16 * kt + 2 * t4);
        ain[kt][2] = *reinterpret_cast<const uint32_t*>(ft + g * MLP_LD1 + 16 * kt + 2 * t4 + 8);
        ain[kt][3] = *reinterpret_cast<const uint32_t*>(ft + (g + 8) * MLP_LD1 + 16 * kt + 2 * t4 + 8);
    }
    uint32_t h1[4][4], h2[4][4], h3[4][4];
    dense_silu<2>(ain, h1, w.W1, MLP_LD1, w.b1, g, t4);
    dense_silu<4>(h1, h2, w.W2, MLP_LDH, w.b2, g, t4);
    dense_silu<4>(h2, h3, w.W3, MLP_LDH, w.b3, g, t4);
    float o[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int kt = 0; kt < 4; ++kt) {
        const unsigned short* wr = w.W4 + g * MLP_LDH + 16 * kt + 2 * t4;
        mma_bf16(o, h3[kt], *reinterpret_cast<const uint32_t*>(wr), *reinterpret_cast<const uint32_t*>(wr + 8));
    }
    if (t4 < 2) {
        out[g][2 * t4] = o[0] + w.b4[2 * t4];
        out[g][2 * t4 + 1] = o[1] + w.b4[2 * t4 + 1];
        out[g + 8][2 * t4] = o[2] + w.b4[2 * t4];
        out[g + 8][2 * t4 + 1] = o[3] + w.b4[2 * t4 + 1];
    }
}

constexpr int MLP_WARPS = 4;

// The fused network alone on raw (unnormalised) features X[n][12]; writes the
// denormalised outputs Y[n][4].  Exposed for numerics tests of mlp_tile.
__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_eval(const MlpDev* wp, const float* X, long long n, float* Y) {
    __shared__ __align__(16) MlpDev w;
    __shared__ __align__(16) unsigned short feat[MLP_WARPS][16 * MLP_LD1];
    __shared__ float outv[MLP_WARPS][16][4];
    {
        const uint4* src = reinterpret_cast<const uint4*>(wp);
        uint4* dst = reinterpret_cast<uint4*>(&w);
        for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    unsigned short* ft = feat[wid];
    const long long ntiles = (n + 15) / 16;
    for (long long tile = (long long)blockIdx.x * MLP_WARPS + wid; tile < ntiles;
         tile += (long long)gridDim.x * MLP_WARPS) {
        const long long r = tile * 16 + (lane & 15);
        if (lane < 16) {
            float f[MLP_IN];
#pragma unroll
            for (int k = 0; k < MLP_IN; ++k) f[k] = r < n ? X[r * MLP_IN + k] : w.in_mu[k];
            store_features(ft + lane * MLP_LD1, f, w);
        }
        __syncwarp();
        mlp_tile(ft, w, outv[wid], g, t4);
        __syncwarp();
        if (lane < 16 && r < n)
            for (int k = 0; k < MLP_OUT; ++k) Y[r * MLP_OUT + k] = mlp_change(w, k, outv[wid][lane][k]);
        __syncwarp();
    }
}

// Surrogate chemistry update: every warp takes 32 cells at a time (one per
// lane for the scalar work, two 16-row tiles for the network).  Per cell:
// the physics predictor; the plain solver's cost estimated from the
// predicted changes (its limiter allows a fraction eps of x_HI, x_HII and E
// per sub-step); cheap cells (estimate <= S.gate sub-steps) go to the plain
// solver's list untouched; the others take the corrected prediction if the
// residual check accepts it, else they join the list too.
__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_chem(const ChemArgs C, const SurrogateArgs S) {
    __shared__ __align__(16) MlpDev w;
    __shared__ __align__(16) unsigned short feat[MLP_WARPS][32 * MLP_LD1];
    __shared__ float outv[MLP_WARPS][32][4];
    {
        const uint4* src = reinterpret_cast<const uint4*>(S.w);
        uint4* dst = reinterpret_cast<uint4*>(&w);
        for (int i = threadIdx.x; i < (int)(sizeof(MlpDev) / 16); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const float y = C.y;
    const float dt = (float)C.dt;
    const float ldt = log10f(dt);
    unsigned accepted = 0;
    const long long ngroups = (C.ncell + 31) / 32;
    unsigned short* ft = feat[wid];
    for (long long grp = (long long)blockIdx.x * MLP_WARPS + wid; grp < ngroups;
         grp += (long long)gridDim.x * MLP_WARPS) {
        const long long c = grp * 32 + lane;
        bool valid = c < C.ncell;
        float nH = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f, T = 1.f, xHeI = 0.f, xHeII = 0.f;
        float G[3] = {0.f, 0.f, 0.f}, H[3] = {0.f, 0.f, 0.f};
        if (valid) {
            nH = C.nH[c];
            a0 = C.xHI[c];
            xHeI = C.xHeI[c];
            xHeII = C.xHeII[c];
            a1 = y * xHeI;
            a2 = y * xHeII;
            T = C.T[c];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                G[q] = C.gamma[q * C.ncell + c];
                H[q] = C.heat[q * C.ncell + c];
            }
            valid = nH > 0.f;   // empty cells are left as they are, as by the plain update
        }
        {
            float f[MLP_IN];
            mlp_features(nH, a0, xHeI, xHeII, T, G, H, ldt, f);
            store_features(ft + lane * MLP_LD1, f, w);
        }
        __syncwarp();
        mlp_tile(ft, w, outv[wid], g, t4);
        mlp_tile(ft + 16 * MLP_LD1, w, outv[wid] + 16, g, t4);
        __syncwarp();
        bool fallback = false;
        if (valid) {
            float p0, p1, p2, pT;
            surrogate_predictor(nH, y, a0, a1, a2, T, G, H, dt, C, p0, p1, p2, pT);
            // sub-steps the plain solver would take, from the predicted changes
            float nest = fabsf(p0 - a0) / (C.eps * fmaxf(fminf(fminf(a0, 1.0f - a0), fminf(p0, 1.0f - p0)), C.xfloor));
            if (!C.isothermal) {
                const float E0 = T * (1.0f + y + (1.0f - a0) + a2 + 2.0f * (y - a1 - a2));
                const float E1 = pT * (1.0f + y + (1.0f - p0) + p2 + 2.0f * (y - p1 - p2));
                nest = fmaxf(nest, fabsf(E1 - E0) / (C.eps * fminf(E0, E1)));
            }
            bool take = false;
            float s0 = 0.f, s1 = 0.f, s2 = 0.f, sT = T;
            if (nest > S.gate) {
                float d[MLP_OUT];
#pragma unroll
                for (int k = 0; k < MLP_OUT; ++k) d[k] = mlp_change(w, k, outv[wid][lane][k]);
                s0 = fminf(fmaxf(p0 + d[0], 0.f), 1.f);
                s1 = fminf(fmaxf(p1 + y * d[1], 0.f), y);
                s2 = fminf(fmaxf(p2 + y * d[2], 0.f), y - s1);
                sT = C.isothermal ? T : fmaxf(pT * exp10f(d[3]), T_FLOOR);
                // a large learned correction marks a step the frozen-coefficient
                // physics misses, and an ionisation front crossing the cell
                // (x_HI or T changing by a large factor within the step) one
                // where the two-half-step check itself is off by ~1e-3: both
                // stay with the plain solver
                const bool small = fabsf(d[0]) <= 4.0f * S.tol_x && fabsf(d[1]) <= 4.0f * S.tol_x &&
                                   fabsf(d[2]) <= 4.0f * S.tol_x && fabsf(d[3]) <= 1.7f * S.tol_e &&
                                   fabsf(s0 - a0) <= 0.1f && sT <= 10.0f * T && T <= 10.0f * sT;
                take = small && surrogate_accept(nH, y, a0, a1, a2, T, s0, s1, s2, sT, G, H, dt, C, S.tol_x, S.tol_e);
            }
            if (take) {
                C.xHI[c] = s0;
                if (y > 0.f) {
                    C.xHeI[c] = s1 / y;
                    C.xHeII[c] = s2 / y;
                }
                C.T[c] = sT;
                accepted++;
            } else {
                fallback = true;
            }
        }
        // the warp's rejected cells join the plain solver's list as one run
        const unsigned fbm = __ballot_sync(0xFFFFFFFFu, fallback);
        if (fbm) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(S.fb_count, (unsigned)__popc(fbm));
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            if (fallback) S.fb_list[base + __popc(fbm & ((1u << lane) - 1u))] = (unsigned)c;
        }
        __syncwarp();
    }
    for (int o = 16; o > 0; o >>= 1) accepted += __shfl_down_sync(0xFFFFFFFFu, accepted, o);
    if (lane == 0 && accepted) atomicAdd(&C.counters[3], (unsigned long long)accepted);
}

// FP32 parameters + normalisation -> padded BF16 device weights (one block)
__global__ void k_pack_mlp(const float* P, const float* norm, MlpDev* out) {
    const float* W1 = P;
    const float* b1 = W1 + MLP_H * MLP_IN;
    const float* W2 = b1 + MLP_H;
    const float* b2 = W2 + MLP_H * MLP_H;
    const float* W3 = b2 + MLP_H;
    const float* b3 = W3 + MLP_H * MLP_H;
    const float* W4 = b3 + MLP_H;
    const float* b4 = W4 + MLP_OUT * MLP_H;
    auto bf = [](float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); };
    for (int i = threadIdx.x; i < MLP_H * MLP_LD1; i += blockDim.x) {
        const int r = i / MLP_LD1, k = i % MLP_LD1, kk = k & 15;   // same W1 for the hi and lo k-tiles
        out->W1[i] = (k < 32 && kk < MLP_IN) ? bf(W1[r * MLP_IN + kk]) : 0;
    }
    for (int i = threadIdx.x; i < MLP_H * MLP_LDH; i += blockDim.x) {
        const int r = i / MLP_LDH, k = i % MLP_LDH;
        out->W2[i] = k < MLP_H ? bf(W2[r * MLP_H + k]) : 0;
        out->W3[i] = k < MLP_H ? bf(W3[r * MLP_H + k]) : 0;
    }
    for (int i = threadIdx.x; i < 8 * MLP_LDH; i += blockDim.x) {
        const int r = i / MLP_LDH, k = i % MLP_LDH;
        out->W4[i] = (r < MLP_OUT && k < MLP_H) ? bf(W4[r * MLP_H + k]) : 0;
    }
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) {
        out->b1[i] = b1[i];
        out->b2[i] = b2[i];
        out->b3[i] = b3[i];
    }
    for (int i = threadIdx.x; i < 8; i += blockDim.x) out->b4[i] = i < MLP_OUT ? b4[i] : 0.f;
    for (int i = threadIdx.x; i < MLP_IN; i += blockDim.x) {
        out->in_mu[i] = norm[i];
        out->in_sd[i] = norm[MLP_IN + i];
    }
    for (int i = threadIdx.x; i < MLP_OUT; i += blockDim.x) {
        out->out_mu[i] = norm[2 * MLP_IN + i];
        out->out_sd[i] = norm[2 * MLP_IN + MLP_OUT + i];
        out->out_s[i] = norm[2 * MLP_IN + 2 * MLP_OUT + i];
    }
}

}  // namespace

cudaError_t launch_chem_surrogate(const ChemArgs& c, const SurrogateArgs& s, cudaStream_t st) {
    // grid-stride over groups of 32 cells; the weights are staged once per block
    long long blocks = ((c.ncell + 31) / 32 + MLP_WARPS - 1) / MLP_WARPS;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_mlp_chem<<<(int)blocks, MLP_WARPS * 32, 0, st>>>(c, s);
    return cudaGetLastError();
}

cudaError_t launch_mlp_eval(const MlpDev* w, const float* X, long long n, float* Y, cudaStream_t s) {
    long long blocks = ((n + 15) / 16 + MLP_WARPS - 1) / MLP_WARPS;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_mlp_eval<<<(int)blocks, MLP_WARPS * 32, 0, s>>>(w, X, n, Y);
    return cudaGetLastError();
}

cudaError_t launch_pack_mlp(const float* params, const float* norm, MlpDev* out, cudaStream_t s) {
    k_pack_mlp<<<1, 256, 0, s>>>(params, norm, out);
    return cudaGetLastError();
}

// Surrogate training targets: the corrections of the converged step (x1, T1)
// to the physics predictor, Y[n][4] = (x_HI' - p0, x_HeI' - p1 / y,
// x_HeII' - p2 / y, log10(T' / pT)).  C holds the start state.
__global__ void k_mlp_targets(const ChemArgs C, const float* x1, const float* T1, float* Y) {
    const float y = C.y, dt = (float)C.dt;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const float nH = C.nH[c];
        const float a0 = C.xHI[c], a1 = y * C.xHeI[c], a2 = y * C.xHeII[c], T = C.T[c];
        float G[3], H[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            G[q] = C.gamma[q * C.ncell + c];
            H[q] = C.heat[q * C.ncell + c];
        }
        float p0, p1, p2, pT;
        surrogate_predictor(nH, y, a0, a1, a2, T, G, H, dt, C, p0, p1, p2, pT);
        Y[c * MLP_OUT + 0] = x1[c] - p0;
        Y[c * MLP_OUT + 1] = y > 0.f ? x1[C.ncell + c] - p1 / y : 0.f;
        Y[c * MLP_OUT + 2] = y > 0.f ? x1[2 * C.ncell + c] - p2 / y : 0.f;
        Y[c * MLP_OUT + 3] = C.isothermal ? 0.f : log10f(T1[c] / pT);
    }
}

cudaError_t launch_mlp_targets(const ChemArgs& c, const float* x1, const float* T1, float* Y, cudaStream_t s) {
    long long blocks = (c.ncell + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_mlp_targets<<<(int)blocks, 256, 0, s>>>(c, x1, T1, Y);
    return cudaGetLastError();
}

// Radiative-transfer time step (Sec. 2.9): per cell dn_HI/dt from the current
// state and the last trace's Gamma_HI (Eq. anninos); out[0] = min of
// eps n_HI / |dn_HI/dt| over cells with n_HI sigma d > 0.5, out[1] = min of
// eps / (sigma d |dn_HI/dt|) over all cells.  Positive floats order like their
// bit patterns, so the minima are integer atomics on them (out preset to +inf).
__global__ void k_rt_timestep(const ChemArgs C, float sigd, float eps, unsigned* out) {
    float dtn = INFINITY, dti = INFINITY;
    const float y = C.y;
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C.ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const float nH = C.nH[c];
        if (!(nH > 0.0f)) continue;
        const float a0 = C.xHI[c], a1 = y * C.xHeI[c], a2 = y * C.xHeII[c];
        const float xe = (1.0f - a0) + a2 + 2.0f * (y - a1 - a2);
        const Coef r = coefficients(C.T[c], C);
        const float ne = nH * xe;
        const float nHI = a0 * nH;
        const float rate = fabsf(r.aH * ne * (nH - nHI) - (C.gamma[c] + r.b0 * ne) * nHI);
        if (!(rate > 0.0f)) continue;
        if (nHI * sigd > 0.5f) dtn = fminf(dtn, eps * nHI / rate);
        dti = fminf(dti, eps / (sigd * rate));
    }
    for (int o = 16; o > 0; o >>= 1) {
        dtn = fminf(dtn, __shfl_down_sync(0xFFFFFFFFu, dtn, o));
        dti = fminf(dti, __shfl_down_sync(0xFFFFFFFFu, dti, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&out[0], __float_as_uint(dtn));
        atomicMin(&out[1], __float_as_uint(dti));
    }
}

cudaError_t launch_rt_timestep(const ChemArgs& c, float sigd, float eps, unsigned* out, cudaStream_t s) {
    long long blocks = (c.ncell + 255) / 256;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    k_rt_timestep<<<(int)blocks, 256, 0, s>>>(c, sigd, eps, out);
    return cudaGetLastError();
}

cudaError_t launch_chem(const ChemArgs& a, cudaStream_t s) {
    long long blocks = (a.ncell + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_chem<<<(int)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace arc
