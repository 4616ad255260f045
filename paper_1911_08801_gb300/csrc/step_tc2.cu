// Persistent, warp-specialised tensor-core as-S_N step (sm_103a).
//
// Work unit: a tile of NT consecutive cells in row-major cell order (tiles may span grid rows),
// all Qp ordinates.  One CTA per SM walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// The artificial in-scattering gain without its diagonal (Sec. 3.2, Eq. (as-S_N equations))
//   D[q][c] = sum_{p != q} K_qp psi~_p(c)
// is one [Mp x Qp] x [Qp x NT] product per tile on tcgen05 (kind::f16, M = 128 ordinates,
// N = NT cells, K = 16, BF16 in, FP32 accumulate in TMEM).  Roles:
//   warp 0      TMEM owner; lane 0 issues the MMAs (k-chunk outer, ordinate block inner) into
//               one of two TMEM accumulator buffers (2 x Mp/128 x NT columns = 512).
//   warp 1      lane 0: TMA producer of the FP32 flux: [NT cells x 64 ordinates] chunks into an
//               SS-stage staging ring.
//   warp 2      lane 0: TMA producer of the kernel-matrix operand G (off-diagonal K in BF16,
//               [128 x 64] chunks, 128-byte swizzle) into an SA-stage ring.
//   warps 3-6   converters: staging chunk -> BF16 B operand (K-major, 128-byte swizzle, written
//               directly in the canonical layout) in an SB-stage ring, and the scalar flux
//               Phi_c = sum_p w_p psi_p(c) accumulated in FP32 over the tile's chunks.
//   warps 7-14  epilogue: drain a TMEM buffer (lane = ordinate, column = cell) and apply upwind
//               transport (Sec. 3.1), collision, isotropic scattering, the source and the
//               generator diagonal:
//                 psi' = psi - a_x (psi - psi_upx) - a_y (psi - psi_upy) - dt sigma_t psi
//                        + dt (sigma_s Phi / sum w + q) + dt sigma_as (D - e psi~)
//               while the MMA of the next tile fills the other buffer.
// SPLIT (BF16X3) keeps BF16 residuals of both operands and issues hi*hi + hi*lo + lo*hi.
//
// Every mbarrier wait is bounded (about 1 s); on expiry the CTA records the event in err_flag,
// all roles stop issuing, the CTA waits briefly for copies and MMAs in flight, frees its tensor
// memory and returns.
#include "assn_internal.h"
#include "tc_ptx.h"

namespace assn {

namespace {

using namespace ptx;

constexpr int kWarps = 15;
constexpr int kThreads2 = kWarps * 32;
constexpr int kAStage = 128 * 64 * 2;   // one [128 x 64] BF16 chunk of G

struct Tc2Args {
    const float* psi;
    float* psi_out;
    const OrdF* ord;
    const CellF* cell;
    const float* w;
    unsigned int* err;
    int nx, ny, Q, Qp, MB, KC, ntiles, ncell;
    int SS, SB, SA, R;
    float dt, dt_sigma_as;
};

constexpr int kEpiWarps = 8;
constexpr int kEpiSlots = 34;     // per chunk and lane: cells fb-1 .. fb+16, then 16 y-neighbours
constexpr int kEpiChunkBytes = kEpiSlots * 32 * 4;
constexpr int kEpiRingMax = 3;    // chunks in flight per epilogue warp (2 or 3)

template <int NT, bool SPLIT>
struct Layout {
    static constexpr int kStg = NT * 256;                       // FP32 staging stage
    static constexpr int kB = NT * 128;                         // BF16 B stage (one of hi / lo)
    static constexpr int kA = kAStage * (SPLIT ? 2 : 1);        // A stage (hi [+ lo])
    int stg, bhi, blo, a, w, phi, epi, bars, end;
    __host__ __device__ Layout(int SS, int SB, int SA, int R, int Qp) {
        stg = 0;
        bhi = stg + SS * kStg;
        blo = bhi + SB * kB;
        a = blo + (SPLIT ? SB * kB : 0);
        w = a + SA * kA;
        phi = w + Qp * 4;                                        // [2][NT] float4 cell coefficients
        epi = phi + 2 * NT * 16;                                 // [8 warps][ring][34][32] floats
        bars = epi + kEpiWarps * R * kEpiChunkBytes;
        // stg_full/empty[SS], bf_full/empty[SB], a_full/empty[SA], tm_full/empty[2], phi_full/empty[2]
        end = bars + 8 * (2 * SS + 2 * SB + 2 * SA + 8) + 16;
    }
};

template <int NT, bool SPLIT>
__global__ void __launch_bounds__(kThreads2, 1)
step_tc2_kernel(const __grid_constant__ CUtensorMap tm_psi, const __grid_constant__ CUtensorMap tm_hi,
                const __grid_constant__ CUtensorMap tm_lo, const Tc2Args a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const Layout<NT, SPLIT> L(a.SS, a.SB, a.SA, a.R, a.Qp);
    float* stg = reinterpret_cast<float*>(base + L.stg);
    unsigned char* bhi = base + L.bhi;
    unsigned char* blo = base + L.blo;
    unsigned char* aring = base + L.a;
    float* wsm = reinterpret_cast<float*>(base + L.w);
    float4* coef = reinterpret_cast<float4*>(base + L.phi);
    float* epi = reinterpret_cast<float*>(base + L.epi);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bars);
    uint64_t* stg_full = bars;
    uint64_t* stg_empty = stg_full + a.SS;
    uint64_t* bf_full = stg_empty + a.SS;
    uint64_t* bf_empty = bf_full + a.SB;
    uint64_t* a_full = bf_empty + a.SB;
    uint64_t* a_empty = a_full + a.SA;
    uint64_t* tm_full = a_empty + a.SA;
    uint64_t* tm_empty = tm_full + 2;
    uint64_t* phi_full = tm_empty + 2;
    uint64_t* phi_empty = phi_full + 2;
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(phi_empty + 2);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int Qp = a.Qp, KC = a.KC, MB = a.MB;

    for (int i = tid; i < Qp; i += blockDim.x) wsm[i] = a.w[i];
    if (tid == 0) {
        for (int s = 0; s < a.SS; ++s) { mbar_init(&stg_full[s], 1); mbar_init(&stg_empty[s], 4); }
        for (int s = 0; s < a.SB; ++s) { mbar_init(&bf_full[s], 4); mbar_init(&bf_empty[s], 1); }
        for (int s = 0; s < a.SA; ++s) { mbar_init(&a_full[s], 1); mbar_init(&a_empty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tm_full[b], 1);
            mbar_init(&tm_empty[b], 8);
            mbar_init(&phi_full[b], 4);
            mbar_init(&phi_empty[b], 8);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) {
        tmem_alloc(tmem_holder, 512);
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------------- MMA issuer
            const uint32_t idesc = idesc_bf16(128, NT);
            int nb = 0, na = 0, it = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
                const int buf = it & 1;
                const uint32_t use = (uint32_t)(it >> 1);
                if (!mbar_wait(&tm_empty[buf], (use & 1u) ^ 1u, abort_flag, a.err, 0x10u)) break;
                tc_fence_after();
                const uint32_t dbase = tmem_base + (uint32_t)(buf * MB * NT);
                bool ok = true;
                for (int kc = 0; kc < KC && ok; ++kc, ++nb) {
                    const int sb = nb % a.SB;
                    if (!mbar_wait(&bf_full[sb], (uint32_t)(nb / a.SB) & 1u, abort_flag, a.err, 0x20u)) { ok = false; break; }
                    tc_fence_after();
                    const uint32_t b_hi = smem_u32(bhi + sb * Layout<NT, SPLIT>::kB);
                    const uint32_t b_lo = smem_u32(blo + sb * Layout<NT, SPLIT>::kB);
                    for (int m = 0; m < MB; ++m, ++na) {
                        const int sa = na % a.SA;
                        if (!mbar_wait(&a_full[sa], (uint32_t)(na / a.SA) & 1u, abort_flag, a.err, 0x40u)) { ok = false; break; }
                        tc_fence_after();
                        const uint32_t a_hi = smem_u32(aring + sa * Layout<NT, SPLIT>::kA);
                        const uint32_t d = dbase + (uint32_t)(m * NT);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk) {
                            const uint64_t ad = sw128_desc(a_hi + kk * 32);
                            const uint64_t bd = sw128_desc(b_hi + kk * 32);
                            mma_bf16(d, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                            if (SPLIT) {
                                mma_bf16(d, ad, sw128_desc(b_lo + kk * 32), idesc, 1u);
                                mma_bf16(d, sw128_desc(a_hi + kAStage + kk * 32), bd, idesc, 1u);
                            }
                        }
                        mma_commit(&a_empty[sa]);
                    }
                    mma_commit(&bf_empty[sb]);
                }
                mma_commit(&tm_full[buf]);
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------------------------------------------------------- flux TMA producer
            // evict-last: the epilogue re-reads these lines (own values and y-neighbours) shortly
            const uint64_t pol = policy_evict_last();
            int ns = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
                bool ok = true;
                for (int kc = 0; kc < KC; ++kc, ++ns) {
                    const int ss = ns % a.SS;
                    if (!mbar_wait(&stg_empty[ss], ((uint32_t)(ns / a.SS) & 1u) ^ 1u, abort_flag, a.err, 0x1u)) { ok = false; break; }
                    mbar_expect_tx(&stg_full[ss], Layout<NT, SPLIT>::kStg);
                    tma_load_2d_hint(stg + (size_t)ss * NT * 64, &tm_psi, &stg_full[ss], kc * 64, tile * NT, pol);
                }
                if (!ok) break;
            }
        }
    } else if (warp == 2) {
        if (lane == 0) {
            // ---------------------------------------------------------------- kernel-matrix TMA producer
            const uint64_t pol = policy_evict_last();   // every tile re-reads G from L2
            int na = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
                bool ok = true;
                for (int kc = 0; kc < KC && ok; ++kc) {
                    for (int m = 0; m < MB; ++m, ++na) {
                        const int sa = na % a.SA;
                        if (!mbar_wait(&a_empty[sa], ((uint32_t)(na / a.SA) & 1u) ^ 1u, abort_flag, a.err, 0x2u)) { ok = false; break; }
                        unsigned char* dst = aring + sa * Layout<NT, SPLIT>::kA;
                        mbar_expect_tx(&a_full[sa], Layout<NT, SPLIT>::kA);
                        tma_load_2d_hint(dst, &tm_hi, &a_full[sa], kc * 64, m * 128, pol);
                        if (SPLIT) tma_load_2d_hint(dst + kAStage, &tm_lo, &a_full[sa], kc * 64, m * 128, pol);
                    }
                }
                if (!ok) break;
            }
        }
    } else if (warp < 7) {
        // -------------------------------------------------------------------- converters
        constexpr int NR = NT / 8;             // rows (cells) per thread
        const int ct = tid - 96;               // 0..127
        const int rsub = ct >> 4;              // 0..7
        const int col4 = ct & 15;              // float4 column within the 64-ordinate chunk
        int ns = 0, nb = 0, it = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
            float part[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) part[i] = 0.0f;
            bool ok = true;
            for (int kc = 0; kc < KC; ++kc, ++ns, ++nb) {
                const int ss = ns % a.SS, sb = nb % a.SB;
                if (!mbar_wait(&stg_full[ss], (uint32_t)(ns / a.SS) & 1u, abort_flag, a.err, 0x100u) ||
                    !mbar_wait(&bf_empty[sb], ((uint32_t)(nb / a.SB) & 1u) ^ 1u, abort_flag, a.err, 0x200u)) {
                    ok = false;
                    break;
                }
                const float4* src = reinterpret_cast<const float4*>(stg + (size_t)ss * NT * 64);
                const float4 w4 = reinterpret_cast<const float4*>(wsm + kc * 64)[col4];
                unsigned char* dhi = bhi + sb * Layout<NT, SPLIT>::kB;
                unsigned char* dlo = blo + sb * Layout<NT, SPLIT>::kB;
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int r = rsub + 8 * i;
                    const float4 v = src[r * 16 + col4];
                    part[i] += w4.x * v.x + w4.y * v.y + w4.z * v.z + w4.w * v.w;
                    uint2 h;
                    h.x = pack_bf16(v.x, v.y);
                    h.y = pack_bf16(v.z, v.w);
                    const int off = (r >> 3) * 1024 + (r & 7) * 128 + ((((col4 >> 1) ^ (r & 7))) << 4) + ((col4 & 1) << 3);
                    *reinterpret_cast<uint2*>(dhi + off) = h;
                    if (SPLIT) {
                        const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.x));
                        const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.y));
                        uint2 l;
                        l.x = pack_bf16(v.x - f0.x, v.y - f0.y);
                        l.y = pack_bf16(v.z - f1.x, v.w - f1.y);
                        *reinterpret_cast<uint2*>(dlo + off) = l;
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&bf_full[sb]);
                    mbar_arrive(&stg_empty[ss]);
                }
            }
            if (!ok) break;
            // Phi of the tile: sum the 16 column partials of each row.
#pragma unroll
            for (int i = 0; i < NR; ++i) {
                float v = part[i];
                v += __shfl_xor_sync(0xffffffffu, v, 8);
                v += __shfl_xor_sync(0xffffffffu, v, 4);
                v += __shfl_xor_sync(0xffffffffu, v, 2);
                v += __shfl_xor_sync(0xffffffffu, v, 1);
                part[i] = v;
            }
            const int buf = it & 1;
            const uint32_t use = (uint32_t)(it >> 1);
            if (!mbar_wait(&phi_empty[buf], (use & 1u) ^ 1u, abort_flag, a.err, 0x400u)) break;
            if (col4 == 0) {
                // per cell: x = 1 - dt sigma_t, y = dt (sigma_s Phi / sum w + q),
                // z = neighbour bits (1 left, 2 right, 4 below, 8 above exist; 16 cell exists)
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int r = rsub + 8 * i;
                    const int f = tile * NT + r;
                    float4 cf = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
                    if (f < a.ncell) {
                        const CellF cl = a.cell[f];
                        const int yy = f / a.nx, xx = f - yy * a.nx;
                        const int bits = (xx > 0 ? 1 : 0) | (xx + 1 < a.nx ? 2 : 0) | (yy > 0 ? 4 : 0) |
                                         (yy + 1 < a.ny ? 8 : 0) | 16;
                        cf = make_float4(1.0f - a.dt * cl.sig_t, a.dt * (cl.sig_s_over_wsum * part[i] + cl.q),
                                         __int_as_float(bits), 0.0f);
                    }
                    coef[buf * NT + r] = cf;
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&phi_full[buf]);
        }
    } else {
        // -------------------------------------------------------------------- epilogue
        // Each warp owns a ring of kEpiRing chunk buffers and prefetches, with cp.async, the flux
        // values its next chunks need (own cells with both x-edge cells, and the upwind y-neighbours)
        // while it computes the current one.  The flux input is read-only during the launch, so the
        // prefetch may run ahead of the MMA.
        float* __restrict__ psi_out = a.psi_out;
        const float* psi = a.psi;
        const int e = warp - 7;
        const int lq = warp & 3;               // TMEM lane quarter this warp may access
        const int half = e >> 2;               // which half of the tile's cells
        const int ncell = a.ncell, nx = a.nx, ny = a.ny;
        constexpr int CPH = NT / 32;           // chunks of 16 cells per half tile
        const int cpt = MB * CPH;              // chunks per tile for this warp
        const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
        const int total = my_tiles * cpt;
        const int R = a.R;
        float* ring = epi + (size_t)e * R * kEpiSlots * 32;

        auto issue = [&](int k) {
            const int t = k / cpt, r = k - t * cpt;
            const int m = r / CPH;
            const int c0 = half * (NT / 2) + (r - m * CPH) * 16;
            const int fb = ((int)blockIdx.x + t * (int)gridDim.x) * NT + c0;
            const int q = m * 128 + lq * 32 + lane;
            const bool qv = q < a.Q;
            float nuy = 0.f;
            if (qv) nuy = a.ord[q].nuy;
            const uint32_t sb = smem_u32(ring + (size_t)(k % R) * kEpiSlots * 32 + lane);
#pragma unroll
            for (int j = 0; j < 18; ++j) {
                const int g = fb - 1 + j;
                const bool ok = qv && g >= 0 && g < ncell;
                cp_async4(sb + j * 128, ok ? psi + (size_t)g * Qp + q : psi, ok ? 4u : 0u);
            }
            int yy = fb / nx, xx = fb - yy * nx;
            const long dyc = nuy > 0.f ? -(long)nx : (long)nx;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int g = fb + i;
                const bool rowok = nuy > 0.f ? yy > 0 : (nuy < 0.f ? yy + 1 < ny : false);
                const bool ok = qv && g < ncell && rowok;
                cp_async4(sb + (18 + i) * 128, ok ? psi + ((long)g + dyc) * Qp + q : psi, ok ? 4u : 0u);
                if (++xx >= nx) { xx -= nx; ++yy; while (xx >= nx) { xx -= nx; ++yy; } }
            }
            cp_async_commit();
        };

        int k_issue = 0;
        for (; k_issue < R - 1 && k_issue < total; ++k_issue) issue(k_issue);
        for (int k = 0; k < total; ++k) {
            if (k_issue < total) issue(k_issue++);
            else cp_async_commit();            // keep one group per iteration
            if (R == 3) cp_async_wait<2>();
            else cp_async_wait<1>();
            const int t = k / cpt, r = k - t * cpt;
            const int m = r / CPH;
            const int c0 = half * (NT / 2) + (r - m * CPH) * 16;
            const int tile = (int)blockIdx.x + t * (int)gridDim.x;
            const int buf = t & 1;
            const uint32_t use = (uint32_t)(t >> 1);
            if (r == 0) {
                int go = 1;
                if (lane == 0)
                    go = mbar_wait(&phi_full[buf], use & 1u, abort_flag, a.err, 0x1000u) &&
                         mbar_wait(&tm_full[buf], use & 1u, abort_flag, a.err, 0x2000u);
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) break;
                tc_fence_after();
            }
            float y[16];
            __syncwarp();
            tmem_ld16(tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * MB * NT + m * NT + c0), y);
            const int fb = tile * NT + c0;
            const int q = m * 128 + lq * 32 + lane;
            if (fb < ncell && q < Qp) {
                float* po = psi_out + (size_t)fb * Qp + q;
                const float4* cbuf = coef + buf * NT + c0;
                if (q >= a.Q) {
#pragma unroll
                    for (int i = 0; i < 16; ++i)
                        if (fb + i < ncell) __stcs(po + (size_t)i * Qp, 0.0f);
                } else {
                    const OrdF o = a.ord[q];
                    const float ax = fabsf(o.nux), ay = fabsf(o.nuy), axy = ax + ay;
                    const int xbit = o.nux > 0.f ? 1 : (o.nux < 0.f ? 2 : 0);
                    const float* sl = ring + (size_t)(k % R) * kEpiSlots * 32 + lane;
#pragma unroll
                    for (int i = 0; i < 16; ++i) {
                        const float4 cf = cbuf[i];
                        const int bits = __float_as_int(cf.z);
                        if (!(bits & 16)) continue;
                        const float sf = sl[(1 + i) * 32];
                        float upx = xbit == 1 ? sl[i * 32] : sl[(i + 2) * 32];
                        upx = (bits & xbit) ? upx : 0.0f;
                        const float upy = sl[(18 + i) * 32];
                        const float st = SPLIT ? sf : __bfloat162float(__float2bfloat16_rn(sf));
                        float out = fmaf(sf, cf.x - axy, cf.y);
                        out = fmaf(ax, upx, out);
                        out = fmaf(ay, upy, out);
                        out = fmaf(a.dt_sigma_as, fmaf(-o.e, st, y[i]), out);
                        __stcs(po + (size_t)i * Qp, out);
                    }
                }
            }
            if (r == cpt - 1) {
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&tm_empty[buf]);
                    mbar_arrive(&phi_empty[buf]);
                }
            }
        }
        cp_async_wait<0>();
    }

    __syncthreads();
    if (*abort_flag) {
        // let copies and MMAs already in flight land before the memory they target goes away
        const uint64_t t0 = globaltimer();
        while (globaltimer() - t0 < 50000ull) __nanosleep(1000);
    }
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
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

bool encode_2d(CUtensorMap* map, CUtensorMapDataType type, const void* ptr, uint64_t inner, uint64_t outer,
               uint64_t row_bytes, uint32_t box_inner, uint32_t box_outer, CUtensorMapSwizzle swz) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {inner, outer};
    const cuuint64_t strides[1] = {row_bytes};
    const cuuint32_t box[2] = {box_inner, box_outer};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, type, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, bool SPLIT>
size_t smem_need(int SS, int SB, int SA, int R, int Qp) {
    return 1024 + (size_t)Layout<NT, SPLIT>(SS, SB, SA, R, Qp).end;
}

size_t smem_for(int NT, bool split, int SS, int SB, int SA, int R, int Qp) {
    switch (NT * 2 + (split ? 1 : 0)) {
        case 64: return smem_need<32, false>(SS, SB, SA, R, Qp);
        case 65: return smem_need<32, true>(SS, SB, SA, R, Qp);
        case 128: return smem_need<64, false>(SS, SB, SA, R, Qp);
        case 129: return smem_need<64, true>(SS, SB, SA, R, Qp);
        case 256: return smem_need<128, false>(SS, SB, SA, R, Qp);
        case 257: return smem_need<128, true>(SS, SB, SA, R, Qp);
        case 512: return smem_need<256, false>(SS, SB, SA, R, Qp);
        default: return smem_need<256, true>(SS, SB, SA, R, Qp);
    }
}

}  // namespace

struct Tc2Plan {
    CUtensorMap tm_hi, tm_lo;
    CUtensorMap tm_psi[4];
    const void* psi_key[4];
    int nkeys;
    int Q, Qp, Mp, MB, KC, NT, SS, SB, SA, R, nx, ny, ncell, ntiles, grid;
    bool split;
    size_t smem;
};

cudaError_t tc2_plan_create(Tc2Plan** out, const __nv_bfloat16* G_hi, const __nv_bfloat16* G_lo, int Q, int Qp,
                            int Mp, int nx, int ny, bool split, int want_nt, int want_stages) {
    *out = nullptr;
    Tc2Plan* p = new Tc2Plan();
    p->Q = Q; p->Qp = Qp; p->Mp = Mp; p->MB = Mp / 128; p->KC = Qp / 64; p->nx = nx; p->ny = ny;
    p->split = split; p->nkeys = 0;
    p->ncell = nx * ny;
    // Tile width: two accumulator buffers of MB x NT columns fill the 512 TMEM columns; narrower
    // when the rings do not fit shared memory.  Ring depths start at 4 / 4 / 4 and the largest
    // ring shrinks (to 2 at least) until the layout fits.
    int nt = 512 / (2 * p->MB);
    if (nt > 256) nt = 256;
    if (want_nt) nt = want_nt;
    const size_t limit = 227 * 1024;
    int SS = 2, SB = 2, SA = 2, R = 2;
    bool fits = false;
    while (!fits) {
        if (nt < 32 || (nt & (nt - 1)) || 2 * p->MB * nt > 512) { delete p; return cudaErrorNotSupported; }
        for (R = kEpiRingMax; R >= 2 && !fits; --R) {
            if (want_stages >= 2) {
                SS = SB = SA = want_stages;
                fits = smem_for(nt, split, SS, SB, SA, R, Qp) <= limit;
            } else if (smem_for(nt, split, 2, 2, 2, R, Qp) <= limit) {
                // deepest balanced rings that fit, then deepen A, the staging ring and B (max 4)
                fits = true;
                SS = SB = SA = 2;
                for (int k = 4; k >= 3; --k)
                    if (smem_for(nt, split, k, k, k, R, Qp) <= limit) { SS = SB = SA = k; break; }
                while (SA < 4 && smem_for(nt, split, SS, SB, SA + 1, R, Qp) <= limit) ++SA;
                while (SS < 4 && smem_for(nt, split, SS + 1, SB, SA, R, Qp) <= limit) ++SS;
                while (SB < 4 && smem_for(nt, split, SS, SB + 1, SA, R, Qp) <= limit) ++SB;
            }
            if (fits) break;
        }
        if (!fits) {
            if (want_nt) { delete p; return cudaErrorNotSupported; }
            nt /= 2;
        }
    }
    p->R = R;
    p->NT = nt;
    p->SS = SS; p->SB = SB; p->SA = SA;
    p->smem = smem_for(nt, split, SS, SB, SA, R, Qp);
    p->ntiles = (p->ncell + nt - 1) / nt;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->grid = p->ntiles < sms ? p->ntiles : sms;
    if (!encode_2d(&p->tm_hi, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, G_hi, Qp, Mp, (uint64_t)Qp * 2, 64, 128,
                   CU_TENSOR_MAP_SWIZZLE_128B) ||
        (split && !encode_2d(&p->tm_lo, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, G_lo, Qp, Mp, (uint64_t)Qp * 2, 64, 128,
                             CU_TENSOR_MAP_SWIZZLE_128B))) {
        delete p;
        return cudaErrorInvalidValue;
    }
    if (!split) p->tm_lo = p->tm_hi;
    *out = p;
    return cudaSuccess;
}

void tc2_plan_destroy(Tc2Plan* p) { delete p; }

void tc2_plan_describe(const Tc2Plan* p, int* tile_cells, int* stages, int* tmem_cols, size_t* smem) {
    if (tile_cells) *tile_cells = p ? p->NT : 0;
    if (stages) *stages = p ? p->SA : 0;
    if (tmem_cols) *tmem_cols = p ? 512 : 0;
    if (smem) *smem = p ? p->smem : 0;
}

static const CUtensorMap* psi_map(Tc2Plan* p, const float* psi) {
    for (int i = 0; i < p->nkeys; ++i)
        if (p->psi_key[i] == psi) return &p->tm_psi[i];
    const int slot = p->nkeys < 4 ? p->nkeys++ : 3;
    if (!encode_2d(&p->tm_psi[slot], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, psi, p->Qp, p->ncell, (uint64_t)p->Qp * 4, 64,
                   p->NT, CU_TENSOR_MAP_SWIZZLE_NONE))
        return nullptr;
    p->psi_key[slot] = psi;
    return &p->tm_psi[slot];
}

template <int NT, bool SPLIT>
static cudaError_t launch2(const Tc2Plan* p, const CUtensorMap* mpsi, const Tc2Args& a, cudaStream_t s) {
    auto kern = step_tc2_kernel<NT, SPLIT>;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    if (r != cudaSuccess) return r;
    kern<<<p->grid, kThreads2, p->smem, s>>>(*mpsi, p->tm_hi, p->tm_lo, a);
    return cudaGetLastError();
}

cudaError_t launch_step_tc2(Tc2Plan* p, const StepArgs<float, OrdF, CellF>& s, const float* w, unsigned int* err_flag,
                            cudaStream_t stream) {
    if (!p) return cudaErrorInvalidValue;
    const CUtensorMap* mpsi = psi_map(p, s.psi);
    if (!mpsi) return cudaErrorInvalidValue;
    Tc2Args a{s.psi, s.psi_out, s.ord, s.cell, w, err_flag, s.nx, s.ny, s.Q, s.Qp, p->MB, p->KC, p->ntiles,
              p->ncell, p->SS, p->SB, p->SA, p->R, s.dt, s.dt_sigma_as};
    switch (p->NT * 2 + (p->split ? 1 : 0)) {
        case 64: return launch2<32, false>(p, mpsi, a, stream);
        case 65: return launch2<32, true>(p, mpsi, a, stream);
        case 128: return launch2<64, false>(p, mpsi, a, stream);
        case 129: return launch2<64, true>(p, mpsi, a, stream);
        case 256: return launch2<128, false>(p, mpsi, a, stream);
        case 257: return launch2<128, true>(p, mpsi, a, stream);
        case 512: return launch2<256, false>(p, mpsi, a, stream);
        default: return launch2<256, true>(p, mpsi, a, stream);
    }
}

}  // namespace assn
