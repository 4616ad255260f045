// Fused as-S_N step with the artificial in-scattering contraction on the 5th-generation tensor
// cores (tcgen05, sm_103a): BF16 operands, FP32 accumulation in tensor memory.
//
// Per CTA: one tile of NT consecutive cells of one grid row, all ordinates.
//   D[q][c] = sum_p G[q][p] psi~[c][p]        (Sec. 3.2: artificial gain without the diagonal)
// is an [Mp x Qp] x [Qp x NT] product issued as tcgen05.mma (M = 128 ordinates, N = NT cells,
// K = 16) with
//   A = G (off-diagonal K in BF16, row q / column p, K-major), streamed by TMA from the
//       L2-resident operand through an S-stage ring of 128 x 64 chunks (128-byte swizzle);
//   B = psi~ (the tile's FP32 flux rounded to BF16, cell-major / ordinate-contiguous = K-major),
//       written by the CTA's threads straight into the canonical 128-byte-swizzled layout while
//       they also reduce the scalar flux Phi = sum_p w_p psi_p in FP32.
// The accumulators (Mp/128 blocks of 128 lanes x NT columns) live in TMEM; the epilogue reads
// them with tcgen05.ld (lane = ordinate, column = cell) and applies upwind transport,
// collision, isotropic scattering, the source and the generator diagonal (Sec. 3.1-3.2):
//   psi' = psi - a_x (psi - psi_upx) - a_y (psi - psi_upy) - dt sigma_t psi
//          + dt (sigma_s Phi / sum w + q) + dt sigma_as (D - e psi~).
// With SPLIT (BF16X3) both operands carry a BF16 residual (hi + lo) and three MMAs per K step
// (hi*hi + hi*lo + lo*hi) give an FP32-accurate contraction.
//
// Every wait on an mbarrier is bounded (about one second of %globaltimer); on expiry the CTA
// records the event in err_flag, stops issuing work, waits (bounded) for what it issued, frees
// its tensor memory and returns.
#include <cuda.h>

#include "assn_internal.h"

namespace assn {

namespace {

constexpr int kThreads = 256;
constexpr int kStageBytes = 128 * 64 * 2;   // one 128-row x 64-column BF16 chunk of G
constexpr uint64_t kWaitNs = 1000000000ull; // bounded waits give up after ~1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait; returns false (and raises the CTA's abort flag) on expiry.
__device__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, unsigned int* err,
                          unsigned int code) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (*abort_flag) return false;
        if (globaltimer() - t0 > kWaitNs) {
            *abort_flag = 1;
            atomicOr(err, code);
            return false;
        }
        __nanosleep(64);
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand in the canonical 128-byte-swizzled layout
// (8-row groups 1024 bytes apart), start address and strides in 16-byte units.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                 // leading-dimension offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // stride between 8-row groups
    d |= (uint64_t)1 << 46;                 // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                 // 128-byte swizzle
    return d;
}

// Instruction descriptor of kind::f16: BF16 x BF16 -> FP32, both operands K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);   // .x = a (low half), .y = b
    return *reinterpret_cast<uint32_t*>(&h);
}

struct TcArgs {
    const float* psi;
    float* psi_out;
    const OrdF* ord;
    const CellF* cell;
    const float* w;        // [Qp] quadrature weights (0 on padding)
    unsigned int* err;
    int nx, ny, Q, Qp, MB, stages, tmem_cols;
    float dt, dt_sigma_as;
};

template <int NT, bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1)
step_tc_kernel(const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo,
               const TcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte alignment (in the shared window) of the swizzled tiles
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int Qp = a.Qp, KC = Qp / 64, S = a.stages;
    unsigned char* B_hi = base;                                       // [KC][NT rows][128 B]
    unsigned char* B_lo = B_hi + (size_t)NT * Qp * 2;                 // SPLIT only
    unsigned char* A0 = B_hi + (size_t)NT * Qp * 2 * (SPLIT ? 2 : 1); // [S][(hi, lo)][16 KB]
    unsigned char* tail = A0 + (size_t)S * kStageBytes * (SPLIT ? 2 : 1);
    uint64_t* full = reinterpret_cast<uint64_t*>(tail);
    uint64_t* empty = full + S;
    uint64_t* done = empty + S;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(done + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
    float* phi = reinterpret_cast<float*>(tmem_holder + 2);           // [NT]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tiles_x = (a.nx + NT - 1) / NT;
    const int j = blockIdx.x / tiles_x;
    const int x0 = (blockIdx.x - j * tiles_x) * NT;
    const int nt = min(NT, a.nx - x0);
    const size_t row = (size_t)j * a.nx;
    const int total_iters = a.MB * KC;

    if (tid == 0) {
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem_base = *tmem_holder;
    const uint32_t stage_tx = kStageBytes * (SPLIT ? 2u : 1u);

    // TMA producer: the first min(S, total) stages need no wait.
    int issued = 0;
    if (warp == 1 && lane == 0) {
        for (; issued < min(S, total_iters); ++issued) {
            const int m = issued / KC, kc = issued - m * KC;
            unsigned char* dst = A0 + (size_t)issued * stage_tx;
            mbar_expect_tx(&full[issued], stage_tx);
            tma_load_2d(dst, &tm_hi, &full[issued], kc * 64, m * 128);
            if (SPLIT) tma_load_2d(dst + kStageBytes, &tm_lo, &full[issued], kc * 64, m * 128);
        }
    }

    // B operand: psi~ of the tile in BF16 (and its residual), swizzled; Phi per cell in FP32.
    {
        int G = 32;                             // lanes per cell: a power of two <= Qp / 8
        while (G > Qp / 8) G >>= 1;
        const int cpw = 32 / G;                 // cells per warp pass
        const int sub = lane / G, g0 = lane - sub * G;
        for (int cb = warp * cpw; cb < NT; cb += (kThreads / 32) * cpw) {
            const int c = cb + sub;
            float part = 0.0f;
            const bool valid = c < nt;
            const float* src = a.psi + (row + x0 + (valid ? c : 0)) * Qp;
            for (int g = g0; g < Qp / 8; g += G) {
                float v[8];
                if (valid) {
                    const float4 u0 = __ldg(reinterpret_cast<const float4*>(src + 8 * g));
                    const float4 u1 = __ldg(reinterpret_cast<const float4*>(src + 8 * g + 4));
                    v[0] = u0.x; v[1] = u0.y; v[2] = u0.z; v[3] = u0.w;
                    v[4] = u1.x; v[5] = u1.y; v[6] = u1.z; v[7] = u1.w;
                    const float4 w0 = __ldg(reinterpret_cast<const float4*>(a.w + 8 * g));
                    const float4 w1 = __ldg(reinterpret_cast<const float4*>(a.w + 8 * g + 4));
                    part += w0.x * v[0] + w0.y * v[1] + w0.z * v[2] + w0.w * v[3] +
                            w1.x * v[4] + w1.y * v[5] + w1.z * v[6] + w1.w * v[7];
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = 0.0f;
                }
                uint4 hi;
                hi.x = pack_bf16(v[0], v[1]); hi.y = pack_bf16(v[2], v[3]);
                hi.z = pack_bf16(v[4], v[5]); hi.w = pack_bf16(v[6], v[7]);
                const int kc = g >> 3, chunk = g & 7;
                const size_t off = (size_t)kc * NT * 128 + (size_t)(c >> 3) * 1024 + (c & 7) * 128 +
                                   ((chunk ^ (c & 7)) << 4);
                *reinterpret_cast<uint4*>(B_hi + off) = hi;
                if (SPLIT) {
                    const __nv_bfloat162* hp = reinterpret_cast<const __nv_bfloat162*>(&hi);
                    float r[8];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float2 f = __bfloat1622float2(hp[i]);
                        r[2 * i] = v[2 * i] - f.x;
                        r[2 * i + 1] = v[2 * i + 1] - f.y;
                    }
                    uint4 lo;
                    lo.x = pack_bf16(r[0], r[1]); lo.y = pack_bf16(r[2], r[3]);
                    lo.z = pack_bf16(r[4], r[5]); lo.w = pack_bf16(r[6], r[7]);
                    *reinterpret_cast<uint4*>(B_lo + off) = lo;
                }
            }
            for (int o = G >> 1; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (g0 == 0 && c < NT) phi[c] = part;
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();

    if (warp == 0 && lane == 0) {
        // MMA issuer.
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t idesc = idesc_bf16(128, NT);
        const uint32_t b_hi = smem_u32(B_hi), b_lo = smem_u32(B_lo);
        for (int it = 0; it < total_iters; ++it) {
            const int s = it % S;
            const uint32_t ph = (uint32_t)(it / S) & 1u;
            if (!mbar_wait(&full[s], ph, abort_flag, a.err, 1u)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int m = it / KC, kc = it - m * KC;
            const uint32_t a_hi = smem_u32(A0 + (size_t)s * stage_tx);
            const uint32_t tmem_d = tmem_base + (uint32_t)(m * NT);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const uint64_t ad = sw128_desc(a_hi + kk * 32);
                const uint64_t bd = sw128_desc(b_hi + kc * NT * 128 + kk * 32);
                mma_bf16(tmem_d, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                if (SPLIT) {
                    const uint64_t bl = sw128_desc(b_lo + kc * NT * 128 + kk * 32);
                    const uint64_t al = sw128_desc(a_hi + kStageBytes + kk * 32);
                    mma_bf16(tmem_d, ad, bl, idesc, 1u);
                    mma_bf16(tmem_d, al, bd, idesc, 1u);
                }
            }
            mma_commit(&empty[s]);
        }
        mma_commit(done);
    } else if (warp == 1 && lane == 0) {
        // TMA producer for the remaining stages.
        for (; issued < total_iters; ++issued) {
            const int s = issued % S;
            const uint32_t ph = ((uint32_t)(issued / S) & 1u) ^ 1u;
            if (!mbar_wait(&empty[s], ph, abort_flag, a.err, 2u)) break;
            const int m = issued / KC, kc = issued - m * KC;
            unsigned char* dst = A0 + (size_t)s * stage_tx;
            mbar_expect_tx(&full[s], stage_tx);
            tma_load_2d(dst, &tm_hi, &full[s], kc * 64, m * 128);
            if (SPLIT) tma_load_2d(dst + kStageBytes, &tm_lo, &full[s], kc * 64, m * 128);
        }
    }
    __syncwarp();

    // Epilogue: wait for the accumulators, then one ordinate per lane, columns = cells.
    // The decision is made once per warp so that tcgen05.ld runs warp-converged.
    int go = 0;
    if (lane == 0) go = mbar_wait(done, 0, abort_flag, a.err, 4u) && !*abort_flag;
    go = __shfl_sync(0xffffffffu, go, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (go) {
        const float* __restrict__ psi = a.psi;
        float* __restrict__ psi_out = a.psi_out;
        const int lq = warp & 3;                 // TMEM lane quarter of this warp
        const int half = warp >> 2;              // which half of the tile's cells
        const int cbeg = half * (NT / 2), cend = cbeg + NT / 2;
        const size_t ystride = (size_t)a.nx * Qp;
        for (int m = 0; m < a.MB; ++m) {
            const int q = m * 128 + lq * 32 + lane;
            const bool qv = q < a.Q;
            const OrdF o = q < Qp ? a.ord[q] : OrdF{0.f, 0.f, 0.f, 0.f};
            const float ax = fabsf(o.nux), ay = fabsf(o.nuy);
            // upwind neighbour offsets (in elements) and whether the neighbour is inside the grid
            const long dx = o.nux > 0.f ? -(long)Qp : (long)Qp;
            const long dy = o.nuy > 0.f ? -(long)ystride : (long)ystride;
            const bool ybound = o.nuy > 0.f ? (j > 0) : (j + 1 < a.ny);
            const bool use_y = o.nuy != 0.f && ybound;
            for (int c0 = cbeg; c0 < cend; c0 += 16) {
                float y[16];
                __syncwarp();
                tmem_ld16(tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(m * NT + c0), y);
                if (!qv) {
                    if (q < Qp) {
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            if (c0 + i < nt) psi_out[(row + x0 + c0 + i) * Qp + q] = 0.0f;
                    }
                    continue;
                }
                float self[16], upx[16], upy[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {       // issue every load of the chunk first
                    const int c = c0 + i;
                    const int x = x0 + c;
                    const bool in = c < nt;
                    const size_t idx = (row + (in ? x : x0)) * Qp + q;
                    self[i] = in ? psi[idx] : 0.0f;
                    const int xn = o.nux > 0.f ? x - 1 : x + 1;
                    upx[i] = (in && o.nux != 0.f && xn >= 0 && xn < a.nx) ? psi[idx + dx] : 0.0f;
                    upy[i] = (in && use_y) ? psi[idx + dy] : 0.0f;
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int c = c0 + i;
                    if (c >= nt) continue;
                    const int x = x0 + c;
                    const CellF cl = a.cell[row + x];
                    const float sf = self[i];
                    const float st = SPLIT ? sf : __bfloat162float(__float2bfloat16_rn(sf));
                    const float out = sf - ax * (sf - upx[i]) - ay * (sf - upy[i]) - a.dt * cl.sig_t * sf +
                                      a.dt * (cl.sig_s_over_wsum * phi[c] + cl.q) +
                                      a.dt_sigma_as * (y[i] - o.e * st);
                    psi_out[(row + x) * Qp + q] = out;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(a.tmem_cols)
                     : "memory");
    }
}

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode() {
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

bool encode_G(CUtensorMap* map, const __nv_bfloat16* G, int Qp, int Mp) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Qp, (cuuint64_t)Mp};
    const cuuint64_t strides[1] = {(cuuint64_t)Qp * 2};
    const cuuint32_t box[2] = {64, 128};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)G, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, bool SPLIT>
size_t smem_bytes(int Qp, int S) {
    return 1024 /*alignment slack*/ + (size_t)NT * Qp * 2 * (SPLIT ? 2 : 1) +
           (size_t)S * kStageBytes * (SPLIT ? 2 : 1) + (2 * S + 1) * 8 + 8 + NT * 4;
}

}  // namespace

struct TcPlan {
    CUtensorMap tm_hi, tm_lo;
    int Q, Qp, Mp, MB, NT, S, tmem_cols, nx, ny;
    bool split;
    size_t smem;
};

void tc_plan_describe(const TcPlan* p, int* tile_cells, int* stages, int* tmem_cols, size_t* smem) {
    if (tile_cells) *tile_cells = p ? p->NT : 0;
    if (stages) *stages = p ? p->S : 0;
    if (tmem_cols) *tmem_cols = p ? p->tmem_cols : 0;
    if (smem) *smem = p ? p->smem : 0;
}

cudaError_t tc_plan_create(TcPlan** out, const __nv_bfloat16* G_hi, const __nv_bfloat16* G_lo, int Q, int Qp,
                           int Mp, int nx, int ny, bool split, int want_nt, int want_stages) {
    *out = nullptr;
    TcPlan* p = new TcPlan();
    p->Q = Q; p->Qp = Qp; p->Mp = Mp; p->MB = Mp / 128; p->nx = nx; p->ny = ny; p->split = split;
    // Tile width: the widest of 128 / 64 / 32 cells (or the requested one) whose accumulators use at
    // most half of the 512 TMEM columns (two CTAs per SM overlap their phases) -- or all of them
    // when nothing smaller fits -- and whose B operand plus a 2-stage A ring fits 200 KB of smem.
    p->NT = 0;
    for (int pass = 0; pass < 2 && p->NT == 0; ++pass) {
        for (int nt : {128, 64, 32}) {
            if (want_nt && nt != want_nt) continue;
            const size_t b = (size_t)nt * Qp * 2 * (split ? 2 : 1);
            const size_t a2 = (size_t)2 * kStageBytes * (split ? 2 : 1);
            const int cap = (pass == 0 && !want_nt) ? 256 : 512;
            if (p->MB * nt <= cap && b + a2 <= 200 * 1024) { p->NT = nt; break; }
        }
    }
    if (p->NT == 0) { delete p; return cudaErrorNotSupported; }
    int cols = p->MB * p->NT;
    int tc = 32;
    while (tc < cols) tc <<= 1;
    p->tmem_cols = tc;
    // Stages: as many as fit in 200 KB, 2..4.
    const size_t b = (size_t)p->NT * Qp * 2 * (split ? 2 : 1);
    p->S = 2;
    while (p->S < 4 && b + (size_t)(p->S + 1) * kStageBytes * (split ? 2 : 1) <= 100 * 1024) p->S++;
    if (want_stages >= 2 && want_stages <= 8 &&
        b + (size_t)want_stages * kStageBytes * (split ? 2 : 1) <= 200 * 1024)
        p->S = want_stages;
    // Residency: never more CTAs per SM than TMEM can hold at once.
    const int max_ctas = 512 / tc;
    size_t sm = 0;
    switch (p->NT * 2 + (split ? 1 : 0)) {
        case 256: sm = smem_bytes<128, false>(Qp, p->S); break;
        case 257: sm = smem_bytes<128, true>(Qp, p->S); break;
        case 128: sm = smem_bytes<64, false>(Qp, p->S); break;
        case 129: sm = smem_bytes<64, true>(Qp, p->S); break;
        case 64: sm = smem_bytes<32, false>(Qp, p->S); break;
        default: sm = smem_bytes<32, true>(Qp, p->S); break;
    }
    const size_t floor_for_residency = 233472 / (max_ctas + 1) - 1024 + 16;
    p->smem = sm > floor_for_residency ? sm : floor_for_residency;
    if (p->smem > 232448) { delete p; return cudaErrorNotSupported; }
    if (!encode_G(&p->tm_hi, G_hi, Qp, Mp) || (split && !encode_G(&p->tm_lo, G_lo, Qp, Mp))) {
        delete p;
        return cudaErrorInvalidValue;
    }
    if (!split) p->tm_lo = p->tm_hi;
    *out = p;
    return cudaSuccess;
}

void tc_plan_destroy(TcPlan* plan) { delete plan; }

template <int NT, bool SPLIT>
static cudaError_t launch_tc(const TcPlan* p, const TcArgs& a, cudaStream_t s) {
    auto kern = step_tc_kernel<NT, SPLIT>;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    if (r != cudaSuccess) return r;
    const int tiles = ((a.nx + NT - 1) / NT) * a.ny;
    kern<<<tiles, kThreads, p->smem, s>>>(p->tm_hi, p->tm_lo, a);
    return cudaGetLastError();
}

cudaError_t launch_step_tc(TcPlan* p, const StepArgs<float, OrdF, CellF>& s, const float* w,
                           unsigned int* err_flag, cudaStream_t stream) {
    if (!p) return cudaErrorInvalidValue;
    TcArgs a{s.psi, s.psi_out, s.ord, s.cell, w, err_flag, s.nx, s.ny, s.Q, s.Qp, p->MB, p->S, p->tmem_cols,
             s.dt, s.dt_sigma_as};
    switch (p->NT * 2 + (p->split ? 1 : 0)) {
        case 256: return launch_tc<128, false>(p, a, stream);
        case 257: return launch_tc<128, true>(p, a, stream);
        case 128: return launch_tc<64, false>(p, a, stream);
        case 129: return launch_tc<64, true>(p, a, stream);
        case 64: return launch_tc<32, false>(p, a, stream);
        default: return launch_tc<32, true>(p, a, stream);
    }
}

}  // namespace assn
