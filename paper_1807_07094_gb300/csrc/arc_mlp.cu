// arc_mlp.cu -- training of the chemistry surrogate on the GPU (sm_103a).
//
// The network (arc_internal.cuh: 12 -> 64 -> 64 -> 64 -> 4, SiLU) is trained
// with mean-squared error on normalised targets.  Every matrix product of the
// forward and backward passes runs on the tensor cores (mma.sync m16n8k16,
// BF16 operands, FP32 accumulation); the master weights and the AdamW moments
// are FP32.  Batch layout is row major: sample b, feature k at [b * ld + k].
//
//   forward   Z_l = A_{l-1} W_l^T + b_l,  A_l = SiLU(Z_l)   (l = 1..3),
//             Yp = A_3 W_4^T + b_4
//   loss      L = mean over samples and the 4 outputs of (Yp - Y)^2
//   backward  dYp = 2 (Yp - Y) / (4 B);  dW_4 = dYp^T A_3;  dA_3 = dYp W_4;
//             dZ_l = dA_l * SiLU'(Z_l);  dW_l = dZ_l^T A_{l-1};  dA_{l-1} = dZ_l W_l
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <string>

#include "arc_internal.cuh"

using namespace arc;

namespace {

constexpr int KP1 = 32;   // layer-1 inputs: BF16 hi (cols 0..15) and lo (16..31) halves, zero padded
constexpr int NP4 = 16;   // output width padded to one 16-row MMA tile (for dW4 = dY^T A3)

__device__ __forceinline__ void mma16816(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
__device__ __forceinline__ uint32_t pk(unsigned short lo, unsigned short hi) {
    return (uint32_t)lo | ((uint32_t)hi << 16);
}
__device__ __forceinline__ unsigned short bf(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// C(m, n) (+)= sum_k A(m, k) B(k, n) with strided BF16 operands
//   A(m, k) = A[m * sam + k * sak],  B(k, n) = B[k * sbk + n * sbn],  C(m, n) = C[m * scm + n * scn]
// M % 16 == 0, N % 8 == 0, K % 16 == 0.  One warp per 16x8 output tile and
// per K chunk of kchunk; chunks are added atomically (C must be zeroed first
// when kchunk < K).
__global__ void k_gemm(int M, int N, int K, int kchunk, const unsigned short* A, long long sam, long long sak,
                       const unsigned short* B, long long sbk, long long sbn, float* C, long long scm,
                       long long scn, int accumulate) {
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int ntn = N / 8, ntm = M / 16;
    const int nk = (K + kchunk - 1) / kchunk;
    if (warp >= (long long)ntm * ntn * nk) return;
    const int kc = (int)(warp % nk);
    const long long t = warp / nk;
    const int m0 = (int)(t / ntn) * 16, n0 = (int)(t % ntn) * 8;
    const int g = lane >> 2, t4 = lane & 3;
    float c[4] = {0.f, 0.f, 0.f, 0.f};
    const int kb = kc * kchunk, ke = min(K, kb + kchunk);
    for (int k0 = kb; k0 < ke; k0 += 16) {
        auto a = [&](int m, int k) { return A[(long long)m * sam + (long long)k * sak]; };
        auto b = [&](int k, int n) { return B[(long long)k * sbk + (long long)n * sbn]; };
        const int ka = k0 + 2 * t4;
        mma16816(c, pk(a(m0 + g, ka), a(m0 + g, ka + 1)), pk(a(m0 + g + 8, ka), a(m0 + g + 8, ka + 1)),
                 pk(a(m0 + g, ka + 8), a(m0 + g, ka + 9)), pk(a(m0 + g + 8, ka + 8), a(m0 + g + 8, ka + 9)),
                 pk(b(ka, n0 + g), b(ka + 1, n0 + g)), pk(b(ka + 8, n0 + g), b(ka + 9, n0 + g)));
    }
    const int rr[4] = {m0 + g, m0 + g, m0 + g + 8, m0 + g + 8};
    const int cc[4] = {n0 + 2 * t4, n0 + 2 * t4 + 1, n0 + 2 * t4, n0 + 2 * t4 + 1};
    for (int i = 0; i < 4; ++i) {
        float* p = C + (long long)rr[i] * scm + (long long)cc[i] * scn;
        if (nk > 1) atomicAdd(p, c[i]);
        else *p = accumulate ? *p + c[i] : c[i];
    }
}

// features (n x 12 FP32, already normalised) -> BF16 n x 32: hi = bf16(v) in
// columns 0..11, lo = bf16(v - hi) in columns 16..27, the rest zero
__global__ void k_pad_inputs(const float* X, long long n, unsigned short* Xb) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * KP1;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / KP1;
        const int k = (int)(i % KP1), kk = k & 15;
        unsigned short out = 0;
        if (kk < MLP_IN) {
            const float v = X[r * MLP_IN + kk];
            const __nv_bfloat16 hi = __float2bfloat16_rn(v);
            out = k < 16 ? __bfloat16_as_ushort(hi) : bf(v - __bfloat162float(hi));
        }
        Xb[i] = out;
    }
}

// Z += bias (row-wise), A = BF16(SiLU(Z)); rows n, width 64
__global__ void k_bias_silu(float* Z, const float* bias, long long n, unsigned short* Ab) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * MLP_H;
         i += (long long)gridDim.x * blockDim.x) {
        const float z = Z[i] + bias[i % MLP_H];
        Z[i] = z;
        Ab[i] = bf(z / (1.0f + expf(-z)));
    }
}

// output: Yp (n x 16) += b4; dYp = 2 (Yp - Y) / (4 n) as BF16 (cols 4..15 zero);
// loss (FP64) += sum (Yp - Y)^2 / (4 n); db4 += column sums of dYp
__global__ void k_out_loss(float* Yp, const float* b4, const float* Y, long long n, unsigned short* dYb,
                           double* loss, float* db4) {
    double part = 0.0;
    float dbl[MLP_OUT] = {0.f, 0.f, 0.f, 0.f};
    const float inv = 1.0f / (float)(MLP_OUT * n);
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * NP4;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / NP4;
        const int k = (int)(i % NP4);
        if (k < MLP_OUT) {
            const float yp = Yp[i] + b4[k];
            Yp[i] = yp;
            const float d = yp - Y[r * MLP_OUT + k];
            part += (double)d * (double)d;
            const float g = 2.0f * d * inv;
            dYb[i] = bf(g);
            dbl[k] += g;
        } else {
            dYb[i] = 0;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        part += __shfl_down_sync(0xFFFFFFFFu, part, o);
        for (int k = 0; k < MLP_OUT; ++k) dbl[k] += __shfl_down_sync(0xFFFFFFFFu, dbl[k], o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(loss, part / (double)(MLP_OUT * n));
        for (int k = 0; k < MLP_OUT; ++k) atomicAdd(&db4[k], dbl[k]);
    }
}

// dZ = dA * SiLU'(Z) (BF16 out), db += column sums (FP32)
__global__ void k_silu_back(const float* dA, const float* Z, long long n, unsigned short* dZb, float* db) {
    __shared__ float acc[MLP_H];
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x) acc[i] = 0.f;
    __syncthreads();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n * MLP_H;
         i += (long long)gridDim.x * blockDim.x) {
        const float z = Z[i];
        const float s = 1.0f / (1.0f + expf(-z));
        const float d = dA[i] * (s * (1.0f + z * (1.0f - s)));
        dZb[i] = bf(d);
        atomicAdd(&acc[i % MLP_H], d);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < MLP_H; i += blockDim.x)
        if (acc[i] != 0.f) atomicAdd(&db[i], acc[i]);
}

// AdamW on the flat FP32 parameters (decoupled weight decay on weights only)
__global__ void k_adamw(float* P, const float* G, float* m, float* v, int np, float lr, float b1, float b2,
                        float wd, float c1, float c2, const unsigned char* is_weight) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const float g = G[i];
        m[i] = b1 * m[i] + (1.0f - b1) * g;
        v[i] = b2 * v[i] + (1.0f - b2) * g * g;
        const float mh = m[i] / c1, vh = v[i] / c2;
        float p = P[i];
        if (is_weight[i]) p -= lr * wd * p;
        P[i] = p - lr * mh / (sqrtf(vh) + 1e-8f);
    }
}

// flat FP32 parameters -> BF16 weight matrices used by the GEMMs
//   W1b [64][32] = [W1 | 0 | W1 | 0] (the same weights for the hi and lo inputs),
//   W2b, W3b [64][64], W4b [16][64] (rows 4..15 zero)
__global__ void k_weights_bf16(const float* P, unsigned short* W1b, unsigned short* W2b, unsigned short* W3b,
                               unsigned short* W4b) {
    const float* W1 = P;
    const float* W2 = W1 + MLP_H * MLP_IN + MLP_H;
    const float* W3 = W2 + MLP_H * MLP_H + MLP_H;
    const float* W4 = W3 + MLP_H * MLP_H + MLP_H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_H * MLP_H; i += gridDim.x * blockDim.x) {
        W2b[i] = bf(W2[i]);
        W3b[i] = bf(W3[i]);
        if (i < MLP_H * KP1) {
            const int r = i / KP1, kk = (i % KP1) & 15;
            W1b[i] = kk < MLP_IN ? bf(W1[r * MLP_IN + kk]) : 0;
        }
        if (i < NP4 * MLP_H) {
            const int r = i / MLP_H;
            W4b[i] = r < MLP_OUT ? bf(W4[i]) : 0;
        }
    }
}

// gradient of W1 from the padded [64][32] product (hi and lo columns summed),
// and of W4 from [16][64]
__global__ void k_unpad_grads(const float* gW1p, const float* gW4p, float* G) {
    float* gW1 = G;
    float* gW4 = G + MLP_H * MLP_IN + MLP_H + 2 * (MLP_H * MLP_H + MLP_H);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_H * MLP_IN; i += gridDim.x * blockDim.x) {
        const float* row = gW1p + (i / MLP_IN) * KP1;
        gW1[i] = row[i % MLP_IN] + row[16 + i % MLP_IN];
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < MLP_OUT * MLP_H; i += gridDim.x * blockDim.x)
        gW4[i] = gW4p[i];
}

// raw surrogate features of n cells (the definition used by the inference kernel)
__global__ void k_features(const float* nH, const float* xHI, const float* xHeI, const float* xHeII,
                           const float* T, const float* gam, const float* heat, float ldt, long long n, float* X) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float G[3] = {gam[i], gam[n + i], gam[2 * n + i]};
        const float H[3] = {heat[i], heat[n + i], heat[2 * n + i]};
        float f[MLP_IN];
        mlp_features(nH[i], xHI[i], xHeI[i], xHeII[i], T[i], G, H, ldt, f);
        for (int k = 0; k < MLP_IN; ++k) X[i * MLP_IN + k] = f[k];
    }
}

int nblk(long long n, int t = 256) {
    long long b = (n + t - 1) / t;
    if (b > 152 * 8) b = 152 * 8;
    return b < 1 ? 1 : (int)b;
}

constexpr int OFF_B1 = MLP_H * MLP_IN;
constexpr int OFF_W2 = OFF_B1 + MLP_H;
constexpr int OFF_B2 = OFF_W2 + MLP_H * MLP_H;
constexpr int OFF_W3 = OFF_B2 + MLP_H;
constexpr int OFF_B3 = OFF_W3 + MLP_H * MLP_H;
constexpr int OFF_W4 = OFF_B3 + MLP_H;
constexpr int OFF_B4 = OFF_W4 + MLP_OUT * MLP_H;
static_assert(OFF_B4 + MLP_OUT == MLP_NPARAMS, "parameter layout");

}  // namespace

struct arc_mlp_trainer {
    cudaStream_t s = nullptr;
    bool own = false;
    int maxb = 0;
    int step = 0;
    float *P = nullptr, *m = nullptr, *v = nullptr, *G = nullptr;
    unsigned char* isw = nullptr;
    unsigned short *W1b = nullptr, *W2b = nullptr, *W3b = nullptr, *W4b = nullptr;
    unsigned short *Xb = nullptr, *A1 = nullptr, *A2 = nullptr, *A3 = nullptr;
    float *Z1 = nullptr, *Z2 = nullptr, *Z3 = nullptr, *Yp = nullptr, *dA = nullptr;
    unsigned short *dY = nullptr, *dZ = nullptr;
    float *gW1p = nullptr, *gW4p = nullptr;
    double* loss = nullptr;
};

extern "C" void arc_mlp_trainer_destroy(arc_mlp_trainer* t);

namespace {

cudaError_t tr_alloc(arc_mlp_trainer* t) {
    const long long B = t->maxb;
    cudaError_t e = cudaSuccess;
    auto al = [&](auto** p, size_t bytes) {
        if (e == cudaSuccess) e = cudaMalloc((void**)p, bytes);
    };
    al(&t->P, MLP_NPARAMS * 4);
    al(&t->m, MLP_NPARAMS * 4);
    al(&t->v, MLP_NPARAMS * 4);
    al(&t->G, MLP_NPARAMS * 4);
    al(&t->isw, MLP_NPARAMS);
    al(&t->W1b, MLP_H * KP1 * 2);
    al(&t->W2b, MLP_H * MLP_H * 2);
    al(&t->W3b, MLP_H * MLP_H * 2);
    al(&t->W4b, NP4 * MLP_H * 2);
    al(&t->Xb, B * KP1 * 2);
    al(&t->A1, B * MLP_H * 2);
    al(&t->A2, B * MLP_H * 2);
    al(&t->A3, B * MLP_H * 2);
    al(&t->Z1, B * MLP_H * 4);
    al(&t->Z2, B * MLP_H * 4);
    al(&t->Z3, B * MLP_H * 4);
    al(&t->Yp, B * NP4 * 4);
    al(&t->dA, B * MLP_H * 4);
    al(&t->dY, B * NP4 * 2);
    al(&t->dZ, B * MLP_H * 2);
    al(&t->gW1p, MLP_H * KP1 * 4);
    al(&t->gW4p, NP4 * MLP_H * 4);
    al(&t->loss, 8);
    return e;
}

// one forward + backward pass over n samples (n % 16 == 0); gradient -> t->G
cudaError_t tr_grad(arc_mlp_trainer* t, const float* X, const float* Y, long long n) {
    cudaStream_t s = t->s;
    const float* P = t->P;
    float* g = t->G;
    cudaError_t e;
    auto gemm = [&](int M, int N, int K, const unsigned short* A, long long sam, long long sak,
                    const unsigned short* B, long long sbk, long long sbn, float* C, long long scm, long long scn) {
        const int kchunk = 1024;   // split K for the weight gradients (K = samples)
        const long long warps = (long long)(M / 16) * (N / 8) * ((K + kchunk - 1) / kchunk);
        k_gemm<<<(int)((warps * 32 + 127) / 128), 128, 0, s>>>(M, N, K, kchunk, A, sam, sak, B, sbk, sbn, C, scm,
                                                              scn, 0);
        return cudaGetLastError();
    };
#define TR_CK(x)                            \
    do {                                    \
        if ((e = (x)) != cudaSuccess) return e; \
    } while (0)
    TR_CK(cudaMemsetAsync(g, 0, MLP_NPARAMS * 4, s));
    TR_CK(cudaMemsetAsync(t->gW1p, 0, MLP_H * KP1 * 4, s));
    TR_CK(cudaMemsetAsync(t->gW4p, 0, NP4 * MLP_H * 4, s));
    TR_CK(cudaMemsetAsync(t->loss, 0, 8, s));
    k_weights_bf16<<<16, 256, 0, s>>>(P, t->W1b, t->W2b, t->W3b, t->W4b);
    k_pad_inputs<<<nblk(n * KP1), 256, 0, s>>>(X, n, t->Xb);
    TR_CK(cudaGetLastError());
    // forward: Z = A_prev W^T (B(k, j) = W[j][k])
    TR_CK(gemm((int)n, MLP_H, KP1, t->Xb, KP1, 1, t->W1b, 1, KP1, t->Z1, MLP_H, 1));
    k_bias_silu<<<nblk(n * MLP_H), 256, 0, s>>>(t->Z1, P + OFF_B1, n, t->A1);
    TR_CK(gemm((int)n, MLP_H, MLP_H, t->A1, MLP_H, 1, t->W2b, 1, MLP_H, t->Z2, MLP_H, 1));
    k_bias_silu<<<nblk(n * MLP_H), 256, 0, s>>>(t->Z2, P + OFF_B2, n, t->A2);
    TR_CK(gemm((int)n, MLP_H, MLP_H, t->A2, MLP_H, 1, t->W3b, 1, MLP_H, t->Z3, MLP_H, 1));
    k_bias_silu<<<nblk(n * MLP_H), 256, 0, s>>>(t->Z3, P + OFF_B3, n, t->A3);
    TR_CK(gemm((int)n, NP4, MLP_H, t->A3, MLP_H, 1, t->W4b, 1, MLP_H, t->Yp, NP4, 1));
    k_out_loss<<<nblk(n * NP4), 256, 0, s>>>(t->Yp, P + OFF_B4, Y, n, t->dY, t->loss, g + OFF_B4);
    TR_CK(cudaGetLastError());
    // output layer: dW4 = dY^T A3 (A(m, k) = dY[k][m]), dA3 = dY W4
    TR_CK(gemm(NP4, MLP_H, (int)n, t->dY, 1, NP4, t->A3, MLP_H, 1, t->gW4p, MLP_H, 1));
    TR_CK(gemm((int)n, MLP_H, NP4, t->dY, NP4, 1, t->W4b, MLP_H, 1, t->dA, MLP_H, 1));
    // hidden layers 3, 2: dZ = dA SiLU'(Z); dW = dZ^T A_prev; dA_prev = dZ W
    k_silu_back<<<nblk(n * MLP_H), 256, 0, s>>>(t->dA, t->Z3, n, t->dZ, g + OFF_B3);
    TR_CK(gemm(MLP_H, MLP_H, (int)n, t->dZ, 1, MLP_H, t->A2, MLP_H, 1, g + OFF_W3, MLP_H, 1));
    TR_CK(gemm((int)n, MLP_H, MLP_H, t->dZ, MLP_H, 1, t->W3b, MLP_H, 1, t->dA, MLP_H, 1));
    k_silu_back<<<nblk(n * MLP_H), 256, 0, s>>>(t->dA, t->Z2, n, t->dZ, g + OFF_B2);
    TR_CK(gemm(MLP_H, MLP_H, (int)n, t->dZ, 1, MLP_H, t->A1, MLP_H, 1, g + OFF_W2, MLP_H, 1));
    TR_CK(gemm((int)n, MLP_H, MLP_H, t->dZ, MLP_H, 1, t->W2b, MLP_H, 1, t->dA, MLP_H, 1));
    // first layer: dZ1 = dA1 SiLU'(Z1); dW1 = dZ1^T X
    k_silu_back<<<nblk(n * MLP_H), 256, 0, s>>>(t->dA, t->Z1, n, t->dZ, g + OFF_B1);
    TR_CK(gemm(MLP_H, KP1, (int)n, t->dZ, 1, MLP_H, t->Xb, KP1, 1, t->gW1p, KP1, 1));
    k_unpad_grads<<<8, 256, 0, s>>>(t->gW1p, t->gW4p, g);
    TR_CK(cudaGetLastError());
#undef TR_CK
    return cudaSuccess;
}

}  // namespace

extern "C" {

arc_status arc_mlp_trainer_create(arc_mlp_trainer** out, int max_batch, void* stream) {
    if (!out || max_batch < 16 || max_batch % 16 || max_batch > (1 << 24)) return ARC_E_INVALID;
    *out = nullptr;
    arc_mlp_trainer* t = new arc_mlp_trainer();
    t->maxb = max_batch;
    t->s = (cudaStream_t)stream;
    if (!t->s) {
        if (cudaStreamCreateWithFlags(&t->s, cudaStreamNonBlocking) != cudaSuccess) {
            delete t;
            return ARC_E_CUDA;
        }
        t->own = true;
    }
    cudaError_t e = tr_alloc(t);
    if (e != cudaSuccess) {
        arc_mlp_trainer_destroy(t);
        return e == cudaErrorMemoryAllocation ? ARC_E_OOM : ARC_E_CUDA;
    }
    // 1 for matrix entries (decayed by AdamW), 0 for biases
    unsigned char isw[MLP_NPARAMS];
    for (int i = 0; i < MLP_NPARAMS; ++i)
        isw[i] = (i < OFF_B1) || (i >= OFF_W2 && i < OFF_B2) || (i >= OFF_W3 && i < OFF_B3) ||
                 (i >= OFF_W4 && i < OFF_B4);
    if (cudaMemcpy(t->isw, isw, MLP_NPARAMS, cudaMemcpyHostToDevice) != cudaSuccess) {
        arc_mlp_trainer_destroy(t);
        return ARC_E_CUDA;
    }
    *out = t;
    return ARC_OK;
}

arc_status arc_mlp_trainer_set_params(arc_mlp_trainer* t, const float* params) {
    if (!t || !params) return ARC_E_INVALID;
    if (cudaMemcpyAsync(t->P, params, MLP_NPARAMS * 4, cudaMemcpyHostToDevice, t->s) != cudaSuccess ||
        cudaMemsetAsync(t->m, 0, MLP_NPARAMS * 4, t->s) != cudaSuccess ||
        cudaMemsetAsync(t->v, 0, MLP_NPARAMS * 4, t->s) != cudaSuccess ||
        cudaStreamSynchronize(t->s) != cudaSuccess)
        return ARC_E_CUDA;
    t->step = 0;
    return ARC_OK;
}

arc_status arc_mlp_trainer_get_params(arc_mlp_trainer* t, float* params) {
    if (!t || !params) return ARC_E_INVALID;
    if (cudaMemcpyAsync(params, t->P, MLP_NPARAMS * 4, cudaMemcpyDeviceToHost, t->s) != cudaSuccess ||
        cudaStreamSynchronize(t->s) != cudaSuccess)
        return ARC_E_CUDA;
    return ARC_OK;
}

arc_status arc_mlp_grad(arc_mlp_trainer* t, const float* X, const float* Y, int n, float* grad, double* loss) {
    if (!t || !X || !Y || n < 16 || n % 16 || n > t->maxb) return ARC_E_INVALID;
    if (tr_grad(t, X, Y, n) != cudaSuccess) return ARC_E_CUDA;
    if (grad && cudaMemcpyAsync(grad, t->G, MLP_NPARAMS * 4, cudaMemcpyDeviceToHost, t->s) != cudaSuccess)
        return ARC_E_CUDA;
    if (loss && cudaMemcpyAsync(loss, t->loss, 8, cudaMemcpyDeviceToHost, t->s) != cudaSuccess) return ARC_E_CUDA;
    if (cudaStreamSynchronize(t->s) != cudaSuccess) return ARC_E_CUDA;
    return ARC_OK;
}

arc_status arc_mlp_train_step(arc_mlp_trainer* t, const float* X, const float* Y, int n, double lr, double wd,
                              double* loss) {
    if (!t || !X || !Y || n < 16 || n % 16 || n > t->maxb || !(lr > 0) || !(wd >= 0)) return ARC_E_INVALID;
    if (tr_grad(t, X, Y, n) != cudaSuccess) return ARC_E_CUDA;
    t->step++;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)t->step), c2 = 1.0f - powf(b2, (float)t->step);
    k_adamw<<<(MLP_NPARAMS + 255) / 256, 256, 0, t->s>>>(t->P, t->G, t->m, t->v, MLP_NPARAMS, (float)lr, b1, b2,
                                                          (float)wd, c1, c2, t->isw);
    if (cudaGetLastError() != cudaSuccess) return ARC_E_CUDA;
    if (loss) {
        if (cudaMemcpyAsync(loss, t->loss, 8, cudaMemcpyDeviceToHost, t->s) != cudaSuccess ||
            cudaStreamSynchronize(t->s) != cudaSuccess)
            return ARC_E_CUDA;
    }
    return ARC_OK;
}

arc_status arc_mlp_eval(const float* params, const float* norm, const float* X, long long n, float* Y,
                        void* stream) {
    if (!params || !norm || !X || !Y || n < 0) return ARC_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    float *dp = nullptr, *dn = nullptr;
    MlpDev* w = nullptr;
    arc_status st = ARC_OK;
    if (cudaMalloc((void**)&dp, MLP_NPARAMS * 4) != cudaSuccess ||
        cudaMalloc((void**)&dn, ARC_MLP_NNORM * 4) != cudaSuccess ||
        cudaMalloc((void**)&w, sizeof(MlpDev)) != cudaSuccess)
        st = ARC_E_OOM;
    if (st == ARC_OK &&
        (cudaMemcpyAsync(dp, params, MLP_NPARAMS * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(dn, norm, ARC_MLP_NNORM * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
         launch_pack_mlp(dp, dn, w, s) != cudaSuccess || launch_mlp_eval(w, X, n, Y, s) != cudaSuccess ||
         cudaStreamSynchronize(s) != cudaSuccess))
        st = ARC_E_CUDA;
    cudaFree(dp);
    cudaFree(dn);
    cudaFree(w);
    return st;
}

arc_status arc_mlp_features(const float* nH, const float* xHI, const float* xHeI, const float* xHeII,
                            const float* T, const float* gamma, const float* heat, double dt, long long n, float* X,
                            void* stream) {
    if (!nH || !xHI || !xHeI || !xHeII || !T || !gamma || !heat || !X || n < 0 || !(dt > 0)) return ARC_E_INVALID;
    k_features<<<nblk(n), 256, 0, (cudaStream_t)stream>>>(nH, xHI, xHeI, xHeII, T, gamma, heat, log10f((float)dt), n, X);
    return cudaGetLastError() == cudaSuccess ? ARC_OK : ARC_E_CUDA;
}

void arc_mlp_trainer_destroy(arc_mlp_trainer* t) {
    if (!t) return;
    if (t->s) cudaStreamSynchronize(t->s);
    void* ptrs[] = {t->P, t->m, t->v, t->G, t->isw, t->W1b, t->W2b, t->W3b, t->W4b, t->Xb, t->A1, t->A2,
                    t->A3, t->Z1, t->Z2, t->Z3, t->Yp, t->dA, t->dY, t->dZ, t->gW1p, t->gW4p, t->loss};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    if (t->own) cudaStreamDestroy(t->s);
    delete t;
}

}  // extern "C"
