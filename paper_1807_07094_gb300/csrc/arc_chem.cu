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
__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

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

// Residual check of a surrogate step (start abundances a0..a2 per H and T;
// prediction s0..s2, sT).  The rate equations of Eq. (anninos) are linear in
// the abundances once n_e and T are fixed; with the coefficients frozen at
// the midpoint of the step (abundances and T averaged between start and
// prediction) they are integrated exactly over dt:
//   HI:  a0' = D - C a0,
//   He:  v' = A v + c for v = (HeI, HeII), HeIII = y - HeI - HeII, whose
//        matrix has real eigenvalues lam1 >= lam2 (the three-state chain is
//        a birth-death process, similar to a symmetric matrix),
// both written v(dt) = v0 + phi(A) (A v0 + c), phi(A) = int_0^dt e^{A t} dt,
// which stays finite as the rates vanish.  The prediction is accepted when
// every abundance agrees with this solution within tol_x (He per He atom)
// and its energy with E0 + dt Edot(midpoint) within tol_e of the energy.

// g(u) = (e^u - 1) / u and its derivative, for u <= 0
__device__ __forceinline__ float g_phi(float u) { return fabsf(u) < 1e-4f ? 1.0f + 0.5f * u : expm1f(u) / u; }
__device__ __forceinline__ float g_phi_d(float u) {
    if (fabsf(u) < 0.1f) return 0.5f + u * (1.0f / 3.0f + u * (0.125f + u * (1.0f / 30.0f + u * (1.0f / 144.0f))));
    return (u * expf(u) - expm1f(u)) / (u * u);
}

__device__ bool surrogate_accept(float nH, float y, float a0, float a1, float a2, float T, float s0, float s1,
                                 float s2, float sT, const float (&G)[3], const float (&H)[3], float dt,
                                 const ChemArgs& C, float tol_x, float tol_e) {
    const float m0 = 0.5f * (a0 + s0), m1 = 0.5f * (a1 + s1), m2 = 0.5f * (a2 + s2);
    const float Tm = 0.5f * (T + sT);
    const float xe = (1.0f - m0) + m2 + 2.0f * (y - m1 - m2);
    const Coef r = coefficients(Tm, C);
    const float ne = nH * xe;
    // hydrogen
    const float CH = G[0] + (r.b0 + r.aH) * ne, DH = r.aH * ne;
    const float e0 = a0 + dt * g_phi(-CH * dt) * (DH - CH * a0);
    if (!(fabsf(e0 - s0) <= tol_x)) return false;
    if (y > 0.0f) {
        // helium chain: A = [[-k1, r2], [k1 - r3, -(k2 + r2 + r3)]], c = (0, r3 y)
        const float k1 = G[1] + r.b1 * ne, k2 = G[2] + r.b2 * ne, r2 = r.a2 * ne, r3 = r.a3 * ne;
        const float A11 = -k1, A12 = r2, A21 = k1 - r3, A22 = -(k2 + r2 + r3);
        const float tr = A11 + A22;
        const float det = k1 * (k2 + r3) + r2 * r3;   // = A11 A22 - A12 A21, all terms >= 0
        const float hd = 0.5f * (A11 - A22);
        const float mu = sqrtf(fmaxf(hd * hd + A12 * A21, 0.0f));
        const float l2 = 0.5f * tr - mu;               // most negative eigenvalue
        const float l1 = l2 < 0.0f ? fminf(det / l2, 0.0f) : 0.0f;
        const float u1 = l1 * dt, u2 = l2 * dt, du = u1 - u2;
        // phi(A) = dt g(u2) I + P1 (A - l2 I), P1 = dt^2 (g(u1) - g(u2)) / (u1 - u2)
        const float um = 0.5f * (u1 + u2);
        const float P1 = dt * dt * (du > 1e-2f * fmaxf(1.0f, fabsf(um)) ? (g_phi(u1) - g_phi(u2)) / du : g_phi_d(um));
        const float p0 = dt * g_phi(u2);
        const float f1 = A11 * a1 + A12 * a2, f2 = A21 * a1 + A22 * a2 + r3 * y;   // v' at the start
        const float e1 = a1 + p0 * f1 + P1 * ((A11 - l2) * f1 + A12 * f2);
        const float e2 = a2 + p0 * f2 + P1 * (A21 * f1 + (A22 - l2) * f2);
        const float th = tol_x * y;
        if (!(fabsf(e1 - s1) <= th) || !(fabsf(e2 - s2) <= th)) return false;
    }
    if (!C.isothermal) {
        const float xe0 = (1.0f - a0) + a2 + 2.0f * (y - a1 - a2);
        const float xe1 = (1.0f - s0) + s2 + 2.0f * (y - s1 - s2);
        const float E0 = 1.5f * KB * T * (1.0f + y + xe0), E1 = 1.5f * KB * sT * (1.0f + y + xe1);
        const float edot = (m0 * H[0] + m1 * H[1] + m2 * H[2]) - cooling_per_h(Tm, nH, m0, m1, m2, xe, r, C);
        if (!(fabsf(E1 - E0 - dt * edot) <= tol_e * fmaxf(E0, E1))) return false;
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

__global__ void __launch_bounds__(MLP_WARPS * 32) k_mlp_chem(const ChemArgs C, const SurrogateArgs S) {
    __shared__ __align__(16) MlpDev w;
    __shared__ __align__(16) unsigned short feat[MLP_WARPS][16 * MLP_LD1];
    __shared__ float outv[MLP_WARPS][16][4];
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
    const long long ntiles = (C.ncell + 15) / 16;
    unsigned short* ft = feat[wid];
    for (long long tile = (long long)blockIdx.x * MLP_WARPS + wid; tile < ntiles;
         tile += (long long)gridDim.x * MLP_WARPS) {
        const long long c = tile * 16 + (lane & 15);
        bool valid = lane < 16 && c < C.ncell;
        float nH = 0.f, a0 = 0.f, a1 = 0.f, a2 = 0.f, T = 1.f;
        float G[3] = {0.f, 0.f, 0.f}, H[3] = {0.f, 0.f, 0.f};
        if (valid) {
            nH = C.nH[c];
            a0 = C.xHI[c];
            a1 = y * C.xHeI[c];
            a2 = y * C.xHeII[c];
            T = C.T[c];
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                G[q] = C.gamma[q * C.ncell + c];
                H[q] = C.heat[q * C.ncell + c];
            }
            valid = nH > 0.f;   // empty cells are left as they are, as by the plain update
        }
        if (lane < 16) {
            float f[MLP_IN];
            mlp_features(nH, a0, valid ? C.xHeI[c] : 0.f, valid ? C.xHeII[c] : 0.f, T, G, H, ldt, f);
            store_features(ft + lane * MLP_LD1, f, w);
        }
        __syncwarp();
        mlp_tile(ft, w, outv[wid], g, t4);
        __syncwarp();
        if (valid) {
            float d[MLP_OUT];
#pragma unroll
            for (int k = 0; k < MLP_OUT; ++k) d[k] = mlp_change(w, k, outv[wid][lane][k]);
            const float s0 = fminf(fmaxf(a0 + d[0], 0.f), 1.f);
            const float s1 = fminf(fmaxf(a1 + y * d[1], 0.f), y);
            const float s2 = fminf(fmaxf(a2 + y * d[2], 0.f), y - s1);
            const float sT = C.isothermal ? T : fmaxf(T * exp10f(d[3]), T_FLOOR);
            if (surrogate_accept(nH, y, a0, a1, a2, T, s0, s1, s2, sT, G, H, dt, C, S.tol_x, S.tol_e)) {
                C.xHI[c] = s0;
                if (y > 0.f) {
                    C.xHeI[c] = s1 / y;
                    C.xHeII[c] = s2 / y;
                }
                C.T[c] = sT;
                accepted++;
            } else {
                const unsigned slot = atomicAdd(S.fb_count, 1u);
                S.fb_list[slot] = (unsigned)c;
            }
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
    long long tiles = (c.ncell + 15) / 16;
    long long blocks = (tiles + MLP_WARPS - 1) / MLP_WARPS;
    if (blocks > 152 * 16) blocks = 152 * 16;
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

cudaError_t launch_chem(const ChemArgs& a, cudaStream_t s) {
    long long blocks = (a.ncell + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    if (blocks < 1) blocks = 1;
    k_chem<<<(int)blocks, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace arc
