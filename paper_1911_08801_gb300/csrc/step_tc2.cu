// Persistent, warp-specialised tensor-core as-S_N step (sm_103a).
//
// Work unit: a tile of NT consecutive cells in row-major cell order (tiles may span grid rows),
// all Qp ordinates.  One CTA per SM walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// The artificial in-scattering gain without its diagonal (Sec. 3.2, Eq. (as-S_N equations))
//   D[q][c] = sum_{p != q} K_qp psi~_p(c)
// is one [Mp x Qp] x [Qp x NT] product per tile on tcgen05 (kind::f16, M = 128 ordinates,
// N = NT cells, K = 16, BF16 in, FP32 accumulate in TMEM).  Roles:
//   warp 0      TMEM owner; lane 0 issues the MMAs (k-chunk outer, ordinate block inner) into
//               one of two TMEM accumulator buffers (2 x Mp/128 x NT columns <= 512).
//   warp 1      lane 0: TMA producer of the FP32 flux: [NT cells x 64 ordinates] chunks into an
//               SS-stage staging ring.
//   warp 2      lane 0: TMA producer of the kernel-matrix operand G (off-diagonal K in BF16,
//               128-byte swizzle) into an SA-stage ring; one 4D request brings the [128 x 64]
//               chunks of MPR ordinate blocks for one k-chunk (a TMA request costs about the same
//               time whatever its size, so requests are made as large as shared memory allows).
//   warps 3-6   converters: staging chunk -> BF16 B operand (K-major, 128-byte swizzle, written
//               directly in the canonical layout) in an SB-stage ring; the scalar flux
//               Phi_c = sum_p w_p psi_p(c) accumulated in FP32 over the tile's chunks, and from it
//               the per-cell coefficients of the update.
//   warps 7-22  epilogue: drain a TMEM buffer (lane = ordinate, column = cell) and apply upwind
//               transport (Sec. 3.1), collision, isotropic scattering, the source and the
//               generator diagonal:
//                 psi' = psi (1 - dt sigma_t - a_x - a_y) + a_x psi_upx + a_y psi_upy
//                        + dt (sigma_s Phi / sum w + q) + dt sigma_as (D - e psi~)
//               while the MMA of the next tile fills the other buffer.  Four warps share each
//               TMEM lane quarter; each keeps the flux values of its next 8-cell chunk in flight
//               (register double buffer).
// SPLIT (BF16X3) keeps BF16 residuals of both operands and issues hi*hi + hi*lo + lo*hi.
// QP > 0 fixes the ordinate stride at compile time (immediate address offsets); QP = 0 reads it
// from the arguments.
//
// Every mbarrier wait is bounded (about 1 s); on expiry the CTA records the event in err_flag,
// all roles stop issuing, the CTA waits briefly for copies and MMAs in flight, frees its tensor
// memory and returns.
#include "assn_internal.h"
#include "tc_ptx.h"

namespace assn {

namespace {

using namespace ptx;

constexpr int kEW = 4;                  // epilogue warps per TMEM lane quarter
constexpr int kCH = 8;                  // cells per epilogue chunk
constexpr int kEpiWarps = 4 * kEW;
constexpr int kWarps = 7 + kEpiWarps;
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
    int SS, SB, SA, MPR;
    float dt, dt_sigma_as;
};

template <int NT, bool SPLIT>
struct Layout {
    static constexpr int kStg = NT * 256;                       // FP32 staging stage
    static constexpr int kB = NT * 128;                         // BF16 B stage (one of hi / lo)
    int kA;                                                     // A stage: MPR blocks (hi [+ lo])
    int stg, bhi, blo, a, w, coef, bars, end;
    __host__ __device__ Layout(int SS, int SB, int SA, int Qp, int MPR) {
        kA = MPR * kAStage * (SPLIT ? 2 : 1);
        stg = 0;
        bhi = stg + SS * kStg;
        blo = bhi + SB * kB;
        a = blo + (SPLIT ? SB * kB : 0);
        w = a + SA * kA;
        coef = w + Qp * 4;                                       // [2][NT] float4 cell coefficients
        bars = coef + 2 * NT * 16;
        // stg_full/empty[SS], bf_full/empty[SB], a_full/empty[SA], tm_full/empty[2], phi_full/empty[2]
        end = bars + 8 * (2 * SS + 2 * SB + 2 * SA + 8) + 16;
    }
};

// Fast path inline, slow (bounded, sleeping) path out of line.
#define WAITB(bar, parity, code) \
    (mbar_try_wait((bar), (parity)) || mbar_wait((bar), (parity), abort_flag, a.err, (code)))

// Ring position: index into an S-deep ring plus the parity of the current pass.
struct Ring {
    int s = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next(int S) {
        if (++s == S) { s = 0; ph ^= 1u; }
    }
};

template <int NT, bool SPLIT, int QP>
__global__ void __launch_bounds__(kThreads2, 1)
step_tc2_kernel(const __grid_constant__ CUtensorMap tm_psi, const __grid_constant__ CUtensorMap tm_hi,
                const __grid_constant__ CUtensorMap tm_lo, const Tc2Args a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const int Qp = QP > 0 ? QP : a.Qp;
    const Layout<NT, SPLIT> L(a.SS, a.SB, a.SA, Qp, a.MPR);
    const int MPR = a.MPR;
    using LT = Layout<NT, SPLIT>;
    float* stg = reinterpret_cast<float*>(base + L.stg);
    unsigned char* bhi = base + L.bhi;
    unsigned char* blo = base + L.blo;
    unsigned char* aring = base + L.a;
    float* wsm = reinterpret_cast<float*>(base + L.w);
    float4* coef = reinterpret_cast<float4*>(base + L.coef);
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
    const int KC = Qp / 64, MB = a.MB;

    for (int i = tid; i < Qp; i += blockDim.x) wsm[i] = a.w[i];
    if (tid == 0) {
        for (int s = 0; s < a.SS; ++s) { mbar_init(&stg_full[s], 1); mbar_init(&stg_empty[s], 4); }
        for (int s = 0; s < a.SB; ++s) { mbar_init(&bf_full[s], 4); mbar_init(&bf_empty[s], 1); }
        for (int s = 0; s < a.SA; ++s) { mbar_init(&a_full[s], 1); mbar_init(&a_empty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tm_full[b], 1);
            mbar_init(&tm_empty[b], kEpiWarps);
            mbar_init(&phi_full[b], 4);
            mbar_init(&phi_empty[b], kEpiWarps);
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
            // descriptors of stage 0 / k-step 0; other stages and k-steps add (byte offset >> 4)
            const uint64_t a0 = sw128_desc(smem_u32(aring));
            const uint64_t b0 = sw128_desc(smem_u32(bhi));
            const uint64_t l0 = sw128_desc(smem_u32(blo));
            Ring rb, ra;
            int it = 0;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
                const int buf = it & 1;
                const uint32_t use = (uint32_t)(it >> 1);
                if (!WAITB(&tm_empty[buf], (use & 1u) ^ 1u, 0x10u)) break;
                tc_fence_after();
                const uint32_t dbase = tmem_base + (uint32_t)(buf * MB * NT);
                bool ok = true;
                for (int kc = 0; kc < KC && ok; ++kc) {
                    if (!WAITB(&bf_full[rb.s], rb.ph, 0x20u)) { ok = false; break; }
                    tc_fence_after();
                    const uint64_t bd0 = b0 + (uint64_t)((rb.s * LT::kB) >> 4);
                    const uint64_t bl0 = l0 + (uint64_t)((rb.s * LT::kB) >> 4);
                    for (int mg = 0; mg < MB; mg += MPR) {
                        if (!WAITB(&a_full[ra.s], ra.ph, 0x40u)) { ok = false; break; }
                        tc_fence_after();
                        const uint64_t as0 = a0 + (uint64_t)((ra.s * L.kA) >> 4);
                        for (int mm = 0; mm < MPR; ++mm) {
                            const uint64_t ad0 = as0 + (uint64_t)((mm * kAStage) >> 4);
                            const uint32_t d = dbase + (uint32_t)((mg + mm) * NT);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = ad0 + (uint64_t)(kk * 2), bd = bd0 + (uint64_t)(kk * 2);
                                mma_bf16(d, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                                if (SPLIT) {
                                    mma_bf16(d, ad, bl0 + (uint64_t)(kk * 2), idesc, 1u);
                                    mma_bf16(d, ad + (uint64_t)((MPR * kAStage) >> 4), bd, idesc, 1u);
                                }
                            }
                        }
                        mma_commit(&a_empty[ra.s]);
                        ra.next(a.SA);
                    }
                    mma_commit(&bf_empty[rb.s]);
                    rb.next(a.SB);
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
            Ring rs;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
                bool ok = true;
                for (int kc = 0; kc < KC; ++kc) {
                    if (!WAITB(&stg_empty[rs.s], rs.ph ^ 1u, 0x1u)) { ok = false; break; }
                    mbar_expect_tx(&stg_full[rs.s], LT::kStg);
                    tma_load_2d_hint(stg + (size_t)rs.s * NT * 64, &tm_psi, &stg_full[rs.s], kc * 64, tile * NT, pol);
                    rs.next(a.SS);
                }
                if (!ok) break;
            }
        }
    } else if (warp == 2) {
        if (lane == 0) {
            // ---------------------------------------------------------------- kernel-matrix TMA producer
            const uint64_t pol = policy_evict_last();   // every tile re-reads G from L2
            Ring ra;
            for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x) {
                bool ok = true;
                for (int kc = 0; kc < KC && ok; ++kc) {
                    for (int mg = 0; mg < MB; mg += MPR) {
                        if (!WAITB(&a_empty[ra.s], ra.ph ^ 1u, 0x2u)) { ok = false; break; }
                        unsigned char* dst = aring + ra.s * L.kA;
                        mbar_expect_tx(&a_full[ra.s], L.kA);
                        tma_load_4d_hint(dst, &tm_hi, &a_full[ra.s], 0, 0, mg, kc, pol);
                        if (SPLIT) tma_load_4d_hint(dst + MPR * kAStage, &tm_lo, &a_full[ra.s], 0, 0, mg, kc, pol);
                        ra.next(a.SA);
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
        Ring rs, rb;
        int it = 0;
        for (int tile = blockIdx.x; tile < a.ntiles; tile += gridDim.x, ++it) {
            float part[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) part[i] = 0.0f;
            bool ok = true;
            for (int kc = 0; kc < KC; ++kc) {
                if (!WAITB(&stg_full[rs.s], rs.ph, 0x100u) || !WAITB(&bf_empty[rb.s], rb.ph ^ 1u, 0x200u)) {
                    ok = false;
                    break;
                }
                const float4* src = reinterpret_cast<const float4*>(stg + (size_t)rs.s * NT * 64);
                const float4 w4 = reinterpret_cast<const float4*>(wsm + kc * 64)[col4];
                unsigned char* dhi = bhi + rb.s * LT::kB;
                unsigned char* dlo = blo + rb.s * LT::kB;
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
                    mbar_arrive(&bf_full[rb.s]);
                    mbar_arrive(&stg_empty[rs.s]);
                }
                rs.next(a.SS);
                rb.next(a.SB);
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
            if (!WAITB(&phi_empty[buf], (use & 1u) ^ 1u, 0x400u)) break;
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
        // Chunks of kCH cells x 32 ordinates.  The flux values of chunk k+1 (own cells, the two
        // x-edge cells, the upwind y-neighbours) are loaded into registers while chunk k is
        // computed.  The flux input is read-only during the launch, so these loads may run ahead
        // of the MMA (and into the next tile).
        const float* __restrict__ psi = a.psi;
        float* __restrict__ psi_out = a.psi_out;
        const int e = warp - 7;
        const int lq = warp & 3;               // TMEM lane quarter this warp may access
        const int grp = e >> 2;                // which part (of kEW) of the tile's cells
        const int ncell = a.ncell, nx = a.nx;
        constexpr int CPH = NT / (kEW * kCH);  // chunks per part of the tile and ordinate block
        const int cpt = MB * CPH;              // chunks per tile for this warp
        const int my_tiles = (a.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
        const int total = my_tiles * cpt;

        // chunk k of this warp: tile index t (within this CTA), ordinate block m, first cell c0
        auto decode = [&](int k, int& t, int& m, int& c0) {
            t = k / cpt;
            const int r = k - t * cpt;
            m = r / CPH;
            c0 = grp * (NT / kEW) + (r - m * CPH) * kCH;
        };
        auto load = [&](int k, float (&s)[kCH], float (&u)[kCH], float& lft, float& rgt) {
            int t, m, c0;
            decode(k, t, m, c0);
            const int fb = ((int)blockIdx.x + t * (int)gridDim.x) * NT + c0;
            const int q = m * 128 + lq * 32 + lane;
            const bool live = q < a.Q && fb < ncell;
            const float nuy = live ? a.ord[q].nuy : 0.0f;
            const float* b = psi + (size_t)(live ? fb : 0) * Qp + (live ? q : 0);
            const bool full = fb + kCH <= ncell;
#pragma unroll
            for (int i = 0; i < kCH; ++i) s[i] = (live && (full || fb + i < ncell)) ? b[i * Qp] : 0.0f;
            // y-neighbour of cell f: below (f - nx) for nuy > 0, above (f + nx) for nuy < 0
            const long dyo = nuy > 0.f ? -(long)nx * Qp : (long)nx * Qp;
            const float* by = b + dyo;
            const bool yall = nuy > 0.f ? fb >= nx : fb + kCH + nx <= ncell;
#pragma unroll
            for (int i = 0; i < kCH; ++i) {
                const int f = fb + i;
                const bool ok = live && nuy != 0.f && (yall || (nuy > 0.f ? f >= nx : f + nx < ncell));
                u[i] = ok ? by[i * Qp] : 0.0f;
            }
            lft = (live && fb >= 1) ? b[-Qp] : 0.0f;
            rgt = (live && fb + kCH < ncell) ? b[kCH * Qp] : 0.0f;
        };
        auto compute = [&](int k, const float (&s)[kCH], const float (&u)[kCH], float lft, float rgt) -> bool {
            int t, m, c0;
            decode(k, t, m, c0);
            const int r = k - t * cpt;
            const int buf = t & 1;
            if (r == 0) {
                const uint32_t use = (uint32_t)(t >> 1);
                int go = 1;
                if (lane == 0)
                    go = WAITB(&phi_full[buf], use & 1u, 0x1000u) && WAITB(&tm_full[buf], use & 1u, 0x2000u);
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) return false;
                tc_fence_after();
            }
            float y[kCH];
            __syncwarp();
            tmem_ld<kCH>(tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * MB * NT + m * NT + c0), y);
            const int fb = ((int)blockIdx.x + t * (int)gridDim.x) * NT + c0;
            const int q = m * 128 + lq * 32 + lane;
            if (fb < ncell && q < Qp) {
                float* po = psi_out + (size_t)fb * Qp + q;
                const float4* cb = coef + buf * NT + c0;
                if (q >= a.Q) {
#pragma unroll
                    for (int i = 0; i < kCH; ++i)
                        if (fb + i < ncell) __stcs(po + i * Qp, 0.0f);
                } else {
                    const OrdF o = a.ord[q];
                    const float ax = fabsf(o.nux), ay = fabsf(o.nuy), axy = ax + ay;
                    const float ge = a.dt_sigma_as * o.e;
                    const int xbit = o.nux > 0.f ? 1 : (o.nux < 0.f ? 2 : 0);
#pragma unroll
                    for (int i = 0; i < kCH; ++i) {
                        const float4 cf = cb[i];
                        const int bits = __float_as_int(cf.z);
                        if (!(bits & 16)) continue;
                        const float sf = s[i];
                        float upx = xbit == 1 ? (i > 0 ? s[i - 1] : lft) : (i < kCH - 1 ? s[i + 1] : rgt);
                        upx = (bits & xbit) ? upx : 0.0f;
                        const float st = SPLIT ? sf : __bfloat162float(__float2bfloat16_rn(sf));
                        float out = fmaf(sf, cf.x - axy, cf.y);
                        out = fmaf(ax, upx, out);
                        out = fmaf(ay, u[i], out);
                        out = fmaf(a.dt_sigma_as, y[i], out);
                        out = fmaf(-ge, st, out);
                        __stcs(po + i * Qp, out);
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
            return true;
        };

        float s0[kCH], u0[kCH], l0 = 0.f, r0 = 0.f, s1[kCH], u1[kCH], l1 = 0.f, r1 = 0.f;
        if (total > 0) load(0, s0, u0, l0, r0);
        for (int k = 0; k < total; k += 2) {
            if (k + 1 < total) load(k + 1, s1, u1, l1, r1);
            if (!compute(k, s0, u0, l0, r0)) break;
            if (k + 1 >= total) break;
            if (k + 2 < total) load(k + 2, s0, u0, l0, r0);
            if (!compute(k + 1, s1, u1, l1, r1)) break;
        }
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

#undef WAITB

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

// 4D view of G [Mp][Qp] BF16: x = column within a 64-column chunk, y = row within a 128-row
// ordinate block, z = ordinate block, w = chunk; box {64, 128, MPR, 1} with 128-byte swizzle lands
// as MPR consecutive canonical [128 x 64] K-major tiles.
bool encode_G4(CUtensorMap* map, const __nv_bfloat16* G, int Qp, int MB, int MPR) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[4] = {64, 128, (cuuint64_t)MB, (cuuint64_t)(Qp / 64)};
    const cuuint64_t strides[3] = {(cuuint64_t)Qp * 2, (cuuint64_t)Qp * 2 * 128, 128};
    const cuuint32_t box[4] = {64, 128, (cuuint32_t)MPR, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16*>(G), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

size_t smem_for(int NT, bool split, int SS, int SB, int SA, int Qp, int MPR) {
    auto need = [&](auto L) { return (size_t)1024 + (size_t)L.end; };
    switch (NT * 2 + (split ? 1 : 0)) {
        case 64: return need(Layout<32, false>(SS, SB, SA, Qp, MPR));
        case 65: return need(Layout<32, true>(SS, SB, SA, Qp, MPR));
        case 128: return need(Layout<64, false>(SS, SB, SA, Qp, MPR));
        case 129: return need(Layout<64, true>(SS, SB, SA, Qp, MPR));
        case 256: return need(Layout<128, false>(SS, SB, SA, Qp, MPR));
        case 257: return need(Layout<128, true>(SS, SB, SA, Qp, MPR));
        case 512: return need(Layout<256, false>(SS, SB, SA, Qp, MPR));
        default: return need(Layout<256, true>(SS, SB, SA, Qp, MPR));
    }
}

}  // namespace

struct Tc2Plan {
    CUtensorMap tm_hi, tm_lo;
    CUtensorMap tm_psi[4];
    const void* psi_key[4];
    int nkeys;
    int Q, Qp, Mp, MB, KC, NT, SS, SB, SA, MPR, nx, ny, ncell, ntiles, grid;
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
    // when the rings do not fit shared memory.  Kernel-matrix requests: as many ordinate blocks per
    // request (MPR) as two stages allow.  Then the deepest balanced staging / B rings that fit (up
    // to 4), then a deeper kernel-matrix ring (up to 4).
    int nt = 512 / (2 * p->MB);
    if (nt > 256) nt = 256;
    if (want_nt) nt = want_nt;
    const size_t limit = 227 * 1024;
    int SS = 2, SB = 2, SA = 2, MPR = 1;
    bool fits = false;
    while (!fits) {
        if (nt < 32 || (nt & (nt - 1)) || 2 * p->MB * nt > 512) { delete p; return cudaErrorNotSupported; }
        for (MPR = p->MB; MPR >= 1 && !fits; MPR /= 2) {
            if (p->MB % MPR) continue;
            if (want_stages >= 2) {
                SS = SB = SA = want_stages;
                fits = smem_for(nt, split, SS, SB, SA, Qp, MPR) <= limit;
            } else if (smem_for(nt, split, 2, 2, 2, Qp, MPR) <= limit) {
                fits = true;
                SS = SB = SA = 2;
                for (int k = 4; k >= 3; --k)
                    if (smem_for(nt, split, k, k, 2, Qp, MPR) <= limit) { SS = SB = k; break; }
                while (SA < 4 && smem_for(nt, split, SS, SB, SA + 1, Qp, MPR) <= limit) ++SA;
            }
            if (fits) break;
        }
        if (!fits) {
            if (want_nt) { delete p; return cudaErrorNotSupported; }
            nt /= 2;
        }
    }
    p->MPR = MPR;
    p->NT = nt;
    p->SS = SS; p->SB = SB; p->SA = SA;
    p->smem = smem_for(nt, split, SS, SB, SA, Qp, MPR);
    p->ntiles = (p->ncell + nt - 1) / nt;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->grid = p->ntiles < sms ? p->ntiles : sms;
    if (!encode_G4(&p->tm_hi, G_hi, Qp, p->MB, MPR) || (split && !encode_G4(&p->tm_lo, G_lo, Qp, p->MB, MPR))) {
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

template <int NT, bool SPLIT, int QP>
static cudaError_t launch2(const Tc2Plan* p, const CUtensorMap* mpsi, const Tc2Args& a, cudaStream_t s) {
    auto kern = step_tc2_kernel<NT, SPLIT, QP>;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    if (r != cudaSuccess) return r;
    kern<<<p->grid, kThreads2, p->smem, s>>>(*mpsi, p->tm_hi, p->tm_lo, a);
    return cudaGetLastError();
}

// Compile-time ordinate strides for the common quadratures (at their automatic tile widths and
// half of them); everything else runs the runtime-stride instance.
template <bool SPLIT>
static cudaError_t dispatch(const Tc2Plan* p, const CUtensorMap* m, const Tc2Args& a, cudaStream_t s) {
    const int key = p->Qp * 1000 + p->NT;
    switch (key) {
        case 512 * 1000 + 64: return launch2<64, SPLIT, 512>(p, m, a, s);
        case 512 * 1000 + 32: return launch2<32, SPLIT, 512>(p, m, a, s);
        case 256 * 1000 + 128: return launch2<128, SPLIT, 256>(p, m, a, s);
        case 256 * 1000 + 64: return launch2<64, SPLIT, 256>(p, m, a, s);
        case 128 * 1000 + 256: return launch2<256, SPLIT, 128>(p, m, a, s);
        case 128 * 1000 + 128: return launch2<128, SPLIT, 128>(p, m, a, s);
        case 64 * 1000 + 256: return launch2<256, SPLIT, 64>(p, m, a, s);
        case 64 * 1000 + 128: return launch2<128, SPLIT, 64>(p, m, a, s);
        default: break;
    }
    switch (p->NT) {
        case 32: return launch2<32, SPLIT, 0>(p, m, a, s);
        case 64: return launch2<64, SPLIT, 0>(p, m, a, s);
        case 128: return launch2<128, SPLIT, 0>(p, m, a, s);
        default: return launch2<256, SPLIT, 0>(p, m, a, s);
    }
}

cudaError_t launch_step_tc2(Tc2Plan* p, const StepArgs<float, OrdF, CellF>& s, const float* w, unsigned int* err_flag,
                            cudaStream_t stream) {
    if (!p) return cudaErrorInvalidValue;
    const CUtensorMap* mpsi = psi_map(p, s.psi);
    if (!mpsi) return cudaErrorInvalidValue;
    Tc2Args a{s.psi, s.psi_out, s.ord, s.cell, w, err_flag, s.nx, s.ny, s.Q, s.Qp, p->MB, p->KC, p->ntiles,
              p->ncell, p->SS, p->SB, p->SA, p->MPR, s.dt, s.dt_sigma_as};
    return p->split ? dispatch<true>(p, mpsi, a, stream) : dispatch<false>(p, mpsi, a, stream);
}

}  // namespace assn
