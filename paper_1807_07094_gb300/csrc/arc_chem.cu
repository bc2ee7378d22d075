// arc_chem.cu -- per-cell H/He ionisation and energy update of libarc (sm_103a).
//
// Sec. 2.7 (Eq. diffeq in the D - C n form of Eq. anninos, backward
// difference, sub-cycled between radiative-transfer steps with the step
// limited to a fraction eps of the change of E, n_HI and n_HII) and Sec. 2.8
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

__device__ __forceinline__ float hg_alpha(float lam) {
    return 2.753e-14f * powf(lam, 1.5f) / powf(1.0f + powf(lam * (1.0f / 2.740f), 0.407f), 2.242f);
}
__device__ __forceinline__ float hg_recool(float T, float lam) {
    return 3.435e-30f * T * powf(lam, 1.970f) / powf(1.0f + powf(lam * (1.0f / 2.250f), 0.376f), 3.720f);
}
__device__ __forceinline__ float dielectronic_shape(float T) {
    return powf(T, -1.5f) * expf(-4.7e5f / T) * (1.0f + 0.3f * expf(-9.4e4f / T));
}

__device__ __forceinline__ Coef coefficients(float T, const ChemArgs& C) {
    const float lHI = 2.0f * TH_HI / T, lHeI = 2.0f * TH_HEI / T, lHeII = 2.0f * TH_HEII / T;
    Coef r;
    r.aH = C.alpha_fixed > 0.0f ? C.alpha_fixed : hg_alpha(lHI);
    r.a2 = 1.26e-14f * powf(lHeI, 0.750f) + 1.90e-3f * dielectronic_shape(T);
    r.a3 = 2.0f * hg_alpha(lHeII);
    if (C.coll_ion) {
        const float t32 = powf(T, -1.5f);
        r.b0 = 21.11f * t32 * expf(-0.5f * lHI) * powf(lHI, -1.089f) /
               powf(1.0f + powf(lHI * (1.0f / 0.354f), 0.874f), 1.101f);
        r.b1 = 32.38f * t32 * expf(-0.5f * lHeI) * powf(lHeI, -1.146f) /
               powf(1.0f + powf(lHeI * (1.0f / 0.416f), 0.987f), 1.056f);
        r.b2 = 19.95f * t32 * expf(-0.5f * lHeII) * powf(lHeII, -1.089f) /
               powf(1.0f + powf(lHeII * (1.0f / 0.553f), 0.735f), 1.275f);
    } else {
        r.b0 = r.b1 = r.b2 = 0.0f;
    }
    return r;
}

// Cooling per hydrogen atom [erg/s]: Lambda / n_H for abundances a0 = HI,
// a1 = HeI, a2 = HeII per H and electrons xe per H.
__device__ __forceinline__ float cooling_per_h(float T, float nH, float a0, float a1, float a2,
                                               float xe, const Coef& r, const ChemArgs& C) {
    const float lHI = 2.0f * TH_HI / T, lHeI = 2.0f * TH_HEI / T, lHeII = 2.0f * TH_HEII / T;
    const float aHII = 1.0f - a0;
    const float a3 = fmaxf(C.y - a1 - a2, 0.0f);          // HeIII per H
    const float nxe = nH * xe;                             // n_e [cm^-3]
    float L = r.b0 * a0 * (KB * TH_HI) + r.b1 * a1 * (KB * TH_HEI) + r.b2 * a2 * (KB * TH_HEII);
    L += hg_recool(T, lHI) * aHII + 1.26e-14f * powf(lHeI, 0.750f) * KB * T * a2 +
         8.0f * hg_recool(T, lHeII) * a3 + 1.24e-13f * dielectronic_shape(T) * a2;
    const float sq = 1.0f + sqrtf(T * 1e-5f);
    L += 7.5e-19f * expf(-118348.0f / T) / sq * a0 + 5.54e-17f * powf(T, -0.397f) * expf(-473638.0f / T) / sq * a2;
    const float lg = log10f(T) - 5.5f;
    const float gff = 1.1f + 0.34f * expf(-lg * lg * (1.0f / 3.0f));
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
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < C.ncell;
         c += (long long)gridDim.x * blockDim.x) {
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

}  // namespace

cudaError_t launch_chem(const ChemArgs& a, cudaStream_t s) {
    long long blocks = (a.ncell + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_chem<<<(int)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace arc
