// Persistent, warp-specialised tensor-core as-S_N step (sm_103a), for one problem or a batch of
// problems of different grid size, ordinate count and kernel width in the same launch.
//
// Work unit: a tile of NT consecutive cells (row-major cell order; tiles may span grid rows) of
// one problem, all its Qp ordinates.  The tiles of all problems form one list; one CTA per SM walks
// it (tile blockIdx.x, blockIdx.x + gridDim.x, ...).  Each problem is described by a ProbDesc in
// device memory (tensor maps, pointers, sizes) and a device step counter: the launch reads the
// flux from buffer (counter & 1), writes buffer (counter & 1) ^ 1, skips problems whose counter
// has reached their target, and the last CTA to finish advances the counters of the problems it
// stepped.  A CUDA graph of such launches therefore steps every solve of an ensemble to its own
// step count.
//
// Per tile, the artificial in-scattering gain without its diagonal (Sec. 3.2, Eq. (as-S_N
// equations))
//   D[q][c] = sum_{p != q} K_qp psi~_p(c)
// is one [Mp x Qp] x [Qp x NT] product on tcgen05 (kind::f16, M = 128 ordinates, N = NT cells,
// K = 16, BF16 in, FP32 accumulate in TMEM).  Roles:
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
//               TMEM lane quarter; the one-pass kernel loads 16-cell chunks of flux values, the
//               split kernel keeps its next 8-cell chunk in flight (register double buffer).
//   Most split forward-Euler kernels and the Heun kernels with tiles of up to 128 cells run 20 warps
//   instead of 23:
//   the G producer is warp 1, lane 1, and warps 2-3 are the converters (epilogue 4-19), which
//   lets each thread hold 96 registers instead of 80.
// SPLIT (BF16X3) keeps BF16 residuals of both operands and issues hi*hi + hi*lo + lo*hi.
// QP > 0 fixes the ordinate stride at compile time (launches whose problems share one of the
// common strides); QP = 0 reads it per problem.
//
// Every mbarrier wait is bounded (about 1 s); on expiry the CTA records the event in err_flag,
// all roles stop issuing, each thread that issued copies or MMAs waits (at most 20 ms, else it
// records kErrUndrained) for its own work to land, the CTA frees its tensor memory and returns,
// and the launch counts no step as taken.
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "assn_internal.h"
#include "tc_ptx.h"

namespace assn {

// Per-problem descriptor (device memory; aligned as its tensor maps require).
struct ProbDesc {
    CUtensorMap tm_psi[2];      // flux buffer b as [ncell][Qp] FP32, box {64, NT}
    CUtensorMap tm_hi, tm_lo;   // kernel-matrix operand, 4D box {64, 128, MPR, 1}
    const float* buf[2];        // flux buffers
    const OrdF* ord;            // [Qp]
    const CellF* cell;          // [ncell]
    const float* w;             // [Qp]
    int* counter;               // steps taken; the launch reads buffer (counter & 1)
    int target;                 // stepped while counter < target
    int nx, ny, ncell, Q, Qp, MB, KC, MPR, ntiles, tile0;
    float dt, dt_sigma_as;
};

namespace {

using namespace ptx;

constexpr int kEW = 4;                  // epilogue warps per TMEM lane quarter
constexpr int kCH = 8;                  // cells per epilogue chunk (double-buffered form)
constexpr int kEpiWarps = 4 * kEW;
constexpr int kAStage = 128 * 64 * 2;   // one [128 x 64] BF16 chunk of G
constexpr int kMaxProbs = 1024;         // problems per launch
constexpr int kParamProbs = 4;          // problems whose tensor maps also travel as kernel parameters

// Tensor maps of one problem, as kernel parameters (the TMA unit reads parameter-space
// descriptors through the constant cache; the copies in ProbDesc serve the other problems).
struct ParamMaps {
    CUtensorMap psi[2], hi, lo;
};

// Scalar parameters of problem 0, read by the epilogue of a one-problem launch (flux buffers
// already resolved by the host from the step parity).
struct OneProb {
    const float* in;
    float* out;
    const OrdF* ord;
    int ncell, nx, Q, Qp, MB;
    float dts;
    const float* keep;                  // Heun stage: out = alpha keep + beta (in + dt L(in))
    float alpha, beta;
};

struct BatchArgs {
    ParamMaps pm[kParamProbs];
    OneProb one;
    int one_fixed;                      // one problem, flux buffers resolved by the host
    const ProbDesc* probs;
    int nprob, total_tiles;
    unsigned int* err;
    unsigned int* ticket;               // CTAs finished; the last one advances the counters
    int SS, SB, SA, MPRmax;
};

template <int NT, bool SPLIT>
struct Layout {
    static constexpr int kStg = NT * 256;                       // FP32 staging stage
    static constexpr int kB = NT * 128;                         // BF16 B stage (one of hi / lo)
    int kA;                                                     // A stage: MPRmax blocks (hi [+ lo])
    int stg, bhi, blo, a, coef, cstage, tparm, pinfo, bars, end;
    __host__ __device__ Layout(int SS, int SB, int SA, int MPRmax) {
        kA = MPRmax * kAStage * (SPLIT ? 2 : 1);
        stg = 0;
        bhi = stg + SS * kStg;
        blo = bhi + SB * kB;
        a = blo + (SPLIT ? SB * kB : 0);
        coef = a + SA * kA;                                      // [2][NT] float4 cell coefficients
        cstage = coef + 2 * NT * 16;                             // [NT] cell constants of the tile
        tparm = cstage + NT * 16;                                // [epilogue warps][2] tile parameters
        pinfo = tparm + kEpiWarps * 2 * 64;                      // [kMaxProbs] first tile, [kMaxProbs] info
        bars = pinfo + kMaxProbs * 8;
        bars = (bars + 7) & ~7;
        // stg_full/empty[SS], bf_full/empty[SB], a_full/empty[SA], tm_full/empty[2], phi_full/empty[2], drain
        end = bars + 8 * (2 * SS + 2 * SB + 2 * SA + 9) + 16;
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

__device__ __forceinline__ float minmod(float a, float b) {
    return a * b > 0.0f ? (fabsf(a) < fabsf(b) ? a : b) : 0.0f;
}

// F_{i+1/2} - F_{i-1/2} in face-value units of the minmod-limited upwind scheme for one ordinate
// along one axis, from the values at i-2 .. i+2 (zero beyond the domain): nu > 0 takes the face
// values psi_i + D_i / 2, nu < 0 takes psi_{i+1} - D_{i+1} / 2 (D: minmod of one-sided differences).
// The lanes of a warp are ordinates of both signs, so both forms are computed from the three slopes
// and one is selected (no divergent branch).
__device__ __forceinline__ float limited_difference(float nu, float m2, float m1, float c0, float p1, float p2) {
    const float dm = minmod(m1 - m2, c0 - m1);   // D_{i-1}
    const float d0 = minmod(c0 - m1, p1 - c0);   // D_i
    const float dp = minmod(p1 - c0, p2 - p1);   // D_{i+1}
    const float pos = (c0 - m1) + 0.5f * (d0 - dm);
    const float neg = (p1 - c0) - 0.5f * (dp - d0);
    return nu > 0.0f ? pos : (nu < 0.0f ? neg : 0.0f);
}

// Problem owning global tile T: the last problem whose first tile is <= T.
__device__ __forceinline__ int find_prob(const int* tile0, int nprob, int T) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile0[mid] <= T) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Warp roles of one kernel instance.  Four converter warps, except in the split forward-Euler
// kernels up to 128-cell tiles and the Heun kernels up to 128-cell tiles: there two converter warps do
// the work and the two TMA producers share warp 1, so that the block has 20 warps and ptxas may give
// each thread 96 registers instead of 80 (the split epilogue keeps two chunks of flux values in
// flight; the Heun epilogue holds the limited stencil of a chunk).  The 128-cell split instance for
// 64 ordinates keeps four converters: with two, its converter rows spill.
template <int NT, bool SPLIT, int QP, bool HEUN>
struct Roles {
    static constexpr bool kTwo = (SPLIT && !HEUN && (NT <= 64 || (NT == 128 && QP != 64))) || (HEUN && NT <= 128);
    static constexpr int kConv = kTwo ? 2 : 4;                             // converter warps
    static constexpr int kConv0 = kConv == 2 ? 2 : 3;                      // first converter warp
    static constexpr int kGWarp = kConv0 - 1, kGLane = kConv == 2 ? 1 : 0; // kernel-matrix producer
    static constexpr int kEpi0 = kConv0 + kConv;                           // first epilogue warp
    static constexpr int kThreads = (kEpi0 + kEpiWarps) * 32;
};

// HEUN: one stage of Heun's method with minmod-limited second-order upwind fluxes (the paper's
// explicit scheme, Sec. 3.1) instead of the forward-Euler first-order step; one-problem launches only.
template <int NT, bool SPLIT, int QP, bool HEUN = false>
__global__ void __launch_bounds__((Roles<NT, SPLIT, QP, HEUN>::kThreads), 1)
step_tc2_kernel(const __grid_constant__ BatchArgs a) {
    using R = Roles<NT, SPLIT, QP, HEUN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const Layout<NT, SPLIT> L(a.SS, a.SB, a.SA, a.MPRmax);
    using LT = Layout<NT, SPLIT>;
    float* stg = reinterpret_cast<float*>(base + L.stg);
    unsigned char* bhi = base + L.bhi;
    unsigned char* blo = base + L.blo;
    unsigned char* aring = base + L.a;
    float4* coef = reinterpret_cast<float4*>(base + L.coef);
    int* s_tile0 = reinterpret_cast<int*>(base + L.pinfo);
    // per problem: bit 0 parity, bit 1 active, bits 8-15 KC, 16-23 MB, 24-31 MPR
    int* s_info = reinterpret_cast<int*>(base + L.pinfo + kMaxProbs * 4);
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
    uint64_t* drain_bar = phi_empty + 2;   // abort path: the MMA issuer's final commit
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(drain_bar + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nprob = a.nprob, total = a.total_tiles;

    for (int i = tid; i < nprob; i += blockDim.x) {
        const ProbDesc& d = a.probs[i];
        const int c = *d.counter;
        s_tile0[i] = d.tile0;
        s_info[i] = (c & 1) | (c < d.target ? 2 : 0) | (d.KC << 8) | (d.MB << 16) | (d.MPR << 24);
    }
    if (tid == 0) {
        for (int s = 0; s < a.SS; ++s) { mbar_init(&stg_full[s], 1); mbar_init(&stg_empty[s], R::kConv); }
        for (int s = 0; s < a.SB; ++s) { mbar_init(&bf_full[s], R::kConv); mbar_init(&bf_empty[s], 1); }
        for (int s = 0; s < a.SA; ++s) { mbar_init(&a_full[s], 1); mbar_init(&a_empty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tm_full[b], 1);
            mbar_init(&tm_empty[b], kEpiWarps);
            mbar_init(&phi_full[b], R::kConv);
            mbar_init(&phi_empty[b], kEpiWarps);
        }
        mbar_init(drain_bar, 1);
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

    // Next active tile of this CTA at or after T (total when none); its problem id in pid.
    auto next_tile = [&](int T, int& pid) -> int {
        for (; T < total; T += gridDim.x) {
            pid = find_prob(s_tile0, nprob, T);
            if (s_info[pid] & 2) return T;
        }
        return total;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------------------------------------------------------- MMA issuer
            const uint32_t idesc = idesc_bf16(128, NT);
            // descriptors of stage 0 / k-step 0; other stages and k-steps add (byte offset >> 4)
            const uint64_t a0 = sw128_desc(smem_u32(aring));
            const uint64_t b0 = sw128_desc(smem_u32(bhi));
            const uint64_t l0 = sw128_desc(smem_u32(blo));
            Ring rb, ra;
            int it = 0, pid = 0;
            for (int T = next_tile(blockIdx.x, pid); T < total; T = next_tile(T + gridDim.x, pid), ++it) {
                const int info = s_info[pid];
                const int KC = QP > 0 ? QP / 64 : (info >> 8) & 255, MB = (info >> 16) & 255, MPR = (info >> 24) & 255;
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
                            const uint32_t dd = dbase + (uint32_t)((mg + mm) * NT);
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = ad0 + (uint64_t)(kk * 2), bd = bd0 + (uint64_t)(kk * 2);
                                mma_bf16(dd, ad, bd, idesc, (kc > 0 || kk > 0) ? 1u : 0u);
                                if (SPLIT) {
                                    mma_bf16(dd, ad, bl0 + (uint64_t)(kk * 2), idesc, 1u);
                                    mma_bf16(dd, ad + (uint64_t)((MPR * kAStage) >> 4), bd, idesc, 1u);
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
            if (*abort_flag) {   // every MMA this thread issued completes before TMEM is freed
                mma_commit(drain_bar);
                if (!mbar_drain(drain_bar, 0u, kDrainNs)) atomicOr(a.err, kErrUndrained);
            }
        }
    } else if (warp == 1 && (lane == 0 || R::kGWarp != 1)) {
        if (lane == 0) {
            // ---------------------------------------------------------------- flux TMA producer
            // evict-last: the epilogue re-reads these lines (own values and y-neighbours) shortly
            const uint64_t pol = policy_evict_last();
            Ring rs;
            uint32_t armed = 0u, apar = 0u;   // slots armed at least once, parity of their last arming
            int pid = 0;
            for (int T = next_tile(blockIdx.x, pid); T < total; T = next_tile(T + gridDim.x, pid)) {
                const int info = s_info[pid];
                const int KC = QP > 0 ? QP / 64 : (info >> 8) & 255;
                const int tile = T - s_tile0[pid];
                const CUtensorMap* map = pid < kParamProbs ? &a.pm[pid].psi[info & 1] : &a.probs[pid].tm_psi[info & 1];
                bool ok = true;
                for (int kc = 0; kc < KC; ++kc) {
                    if (!WAITB(&stg_empty[rs.s], rs.ph ^ 1u, 0x1u)) { ok = false; break; }
                    mbar_expect_tx(&stg_full[rs.s], LT::kStg);
                    tma_load_2d_hint(stg + (size_t)rs.s * NT * 64, map, &stg_full[rs.s], kc * 64, tile * NT, pol);
                    armed |= 1u << rs.s;
                    apar = (apar & ~(1u << rs.s)) | (rs.ph << rs.s);
                    rs.next(a.SS);
                }
                if (!ok) break;
            }
            if (*abort_flag)   // copies in flight land before the staging ring is released
                for (int s2 = 0; s2 < a.SS; ++s2)
                    if (((armed >> s2) & 1u) && !mbar_drain(&stg_full[s2], (apar >> s2) & 1u, kDrainNs))
                        atomicOr(a.err, kErrUndrained);
        }
    } else if (warp == R::kGWarp) {
        if (lane == R::kGLane) {
            // ---------------------------------------------------------------- kernel-matrix TMA producer
            const uint64_t pol = policy_evict_last();   // every tile re-reads G from L2
            Ring ra;
            uint32_t armed = 0u, apar = 0u;
            int pid = 0;
            for (int T = next_tile(blockIdx.x, pid); T < total; T = next_tile(T + gridDim.x, pid)) {
                const int info = s_info[pid];
                const int KC = QP > 0 ? QP / 64 : (info >> 8) & 255, MB = (info >> 16) & 255, MPR = (info >> 24) & 255;
                const int bytes = MPR * kAStage * (SPLIT ? 2 : 1);
                const CUtensorMap* mhi = pid < kParamProbs ? &a.pm[pid].hi : &a.probs[pid].tm_hi;
                const CUtensorMap* mlo = pid < kParamProbs ? &a.pm[pid].lo : &a.probs[pid].tm_lo;
                bool ok = true;
                for (int kc = 0; kc < KC && ok; ++kc) {
                    for (int mg = 0; mg < MB; mg += MPR) {
                        if (!WAITB(&a_empty[ra.s], ra.ph ^ 1u, 0x2u)) { ok = false; break; }
                        unsigned char* dst = aring + ra.s * L.kA;
                        mbar_expect_tx(&a_full[ra.s], bytes);
                        tma_load_4d_hint(dst, mhi, &a_full[ra.s], 0, 0, mg, kc, pol);
                        if (SPLIT) tma_load_4d_hint(dst + MPR * kAStage, mlo, &a_full[ra.s], 0, 0, mg, kc, pol);
                        armed |= 1u << ra.s;
                        apar = (apar & ~(1u << ra.s)) | (ra.ph << ra.s);
                        ra.next(a.SA);
                    }
                }
                if (!ok) break;
            }
            if (*abort_flag)
                for (int s2 = 0; s2 < a.SA; ++s2)
                    if (((armed >> s2) & 1u) && !mbar_drain(&a_full[s2], (apar >> s2) & 1u, kDrainNs))
                        atomicOr(a.err, kErrUndrained);
        }
    } else if (warp < R::kEpi0) {
        // -------------------------------------------------------------------- converters
        constexpr int RS = 2 * R::kConv;       // row stride: rows handled by one column of threads
        constexpr int NR = NT / RS;            // rows (cells) per thread
        const int ct = tid - 32 * R::kConv0;   // 0 .. 32 kConv - 1
        const int rsub = ct >> 4;              // 0 .. RS - 1
        const int col4 = ct & 15;              // float4 column within the 64-ordinate chunk
        // Problem fields are refetched only when the tile's problem changes; the weights of the
        // next chunk (across tile ends) and the cell constants of the tile (cp.async into this
        // thread's own rows of cstage) are requested ahead of use.
        CellF* cstage = reinterpret_cast<CellF*>(base + L.cstage);
        Ring rs, rb;
        int it = 0, pid = 0, cpid = -1;
        const float4* wp = nullptr;
        const CellF* cellp = nullptr;
        int nx = 1, ny = 1, ncell = 0;
        float dt = 0.0f;
        float4 wn = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int T = next_tile(blockIdx.x, pid); T < total; T = next_tile(T + gridDim.x, pid), ++it) {
            if (pid != cpid) {
                const ProbDesc& d = a.probs[pid];
                wp = reinterpret_cast<const float4*>(d.w) + col4;
                cellp = d.cell;
                nx = d.nx;
                ny = d.ny;
                ncell = d.ncell;
                dt = d.dt;
                wn = __ldg(wp);
                cpid = pid;
            }
            const int KC = QP > 0 ? QP / 64 : (s_info[pid] >> 8) & 255;
            const int tile = T - s_tile0[pid];
            if (col4 == 0) {
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int r = rsub + RS * i;
                    const int f = tile * NT + r;
                    if (f < ncell) cp_async16(smem_u32(cstage + r), cellp + f, 16u);
                }
                cp_async_commit();
            }
            float part[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) part[i] = 0.0f;
            bool ok = true;
            for (int kc = 0; kc < KC; ++kc) {
                const float4 w4 = wn;
                wn = __ldg(wp + (kc + 1 < KC ? kc + 1 : 0) * 16);
                if (!WAITB(&stg_full[rs.s], rs.ph, 0x100u) || !WAITB(&bf_empty[rb.s], rb.ph ^ 1u, 0x200u)) {
                    ok = false;
                    break;
                }
                const float4* src = reinterpret_cast<const float4*>(stg + (size_t)rs.s * NT * 64);
                unsigned char* dhi = bhi + rb.s * LT::kB;
                unsigned char* dlo = blo + rb.s * LT::kB;
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int r = rsub + RS * i;
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
                // z = neighbour bits (1 left, 2 right, 4 below, 8 above exist; 16 cell exists; 32 / 64 the cells
                // two to the left / right exist)
                cp_async_wait<0>();
#pragma unroll
                for (int i = 0; i < NR; ++i) {
                    const int r = rsub + RS * i;
                    const int f = tile * NT + r;
                    float4 cf = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
                    if (f < ncell) {
                        const CellF cl = cstage[r];
                        const int yy = f / nx, xx = f - yy * nx;
                        const int bits = (xx > 0 ? 1 : 0) | (xx + 1 < nx ? 2 : 0) | (yy > 0 ? 4 : 0) |
                                         (yy + 1 < ny ? 8 : 0) | 16 | (xx > 1 ? 32 : 0) | (xx + 2 < nx ? 64 : 0);
                        cf = make_float4(1.0f - dt * cl.sig_t, dt * (cl.sig_s_over_wsum * part[i] + cl.q),
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
        // Chunks of kCHe cells x 32 ordinates.  The warp's time per chunk is set by the latency of
        // its flux loads (own cells, the two x-edge cells, the upwind y-neighbours), so what counts
        // is how many bytes a warp keeps in flight: the one-pass kernel loads 16-cell chunks and
        // waits for them (one buffer); the split kernel, whose MMA work is three times longer,
        // keeps 8-cell chunks double-buffered (the next chunk's loads in flight while the current
        // one is computed).  The flux input is read-only during the launch, so loads may run ahead
        // of the MMA (and into the next tile).
        const int e = warp - R::kEpi0;
        const int lq = warp & 3;               // TMEM lane quarter this warp may access
        const int grp = e >> 2;                // which part (of kEW) of the tile's cells
        constexpr bool kOneBuf = HEUN || (!SPLIT && NT / kEW >= 16);
        constexpr int kCHe = HEUN ? kCH : (kOneBuf ? 16 : kCH);
        constexpr int CPH = NT / (kEW * kCHe);  // chunks per part of the tile and ordinate block

        // Position of a chunk: global tile T of problem pid, the it-th active tile of this CTA,
        // chunk r within that tile (cpt chunks per tile).
        struct Pos {
            int T, pid, it, r, cpt;
        };
        // Problem parameters of a tile as the chunk code uses them.
        struct alignas(16) TileP {
            const float* in;
            float* out;
            const OrdF* ord;
            const float* keep;                 // Heun stage 2: psi^n (the output buffer); else unused
            int fb0, ncell, nx, Q, Qp;
            float dts, alpha, beta;            // Heun: out = alpha keep + beta (in + dt L(in))
        };
        static_assert(sizeof(TileP) <= 64, "tile parameter slot");

        // Flux loads of chunk r (ordinate block m = r / CPH) of a tile into registers.
        auto load = [&](const TileP& t, int r, float (&s)[kCHe], float (&u)[kCHe], float& lft, float& rgt) {
            const int Qp = QP > 0 ? QP : t.Qp;
            const int m = r / CPH;
            const int c0 = grp * (NT / kEW) + (r - m * CPH) * kCHe;
            const int ncell = t.ncell, nx = t.nx;
            const int fb = t.fb0 + c0;
            const int q = m * 128 + lq * 32 + lane;
            const bool live = q < t.Q && fb < ncell;
            const float nuy = live ? __ldg(&t.ord[q].nuy) : 0.0f;
            const float* b = t.in + (size_t)(live ? fb : 0) * Qp + (live ? q : 0);
            const bool full = fb + kCHe <= ncell;
#pragma unroll
            for (int i = 0; i < kCHe; ++i) s[i] = (live && (full || fb + i < ncell)) ? __ldg(b + i * Qp) : 0.0f;
            // y-neighbour of cell f: below (f - nx) for nuy > 0, above (f + nx) for nuy < 0
            const long dyo = nuy > 0.f ? -(long)nx * Qp : (long)nx * Qp;
            const float* by = b + dyo;
            const bool yall = nuy > 0.f ? fb >= nx : fb + kCHe + nx <= ncell;
#pragma unroll
            for (int i = 0; i < kCHe; ++i) {
                const int f = fb + i;
                const bool ok = live && nuy != 0.f && (yall || (nuy > 0.f ? f >= nx : f + nx < ncell));
                u[i] = ok ? __ldg(by + i * Qp) : 0.0f;
            }
            lft = (live && fb >= 1) ? __ldg(b - Qp) : 0.0f;
            rgt = (live && fb + kCHe < ncell) ? __ldg(b + kCHe * Qp) : 0.0f;
        };
        // Update of chunk r of the it-th tile of this CTA (cpt chunks per tile); false on abort.
        auto compute = [&](const TileP& t, int it, int r, int cpt, const float (&s)[kCHe], const float (&u)[kCHe],
                           float lft, float rgt) -> bool {
            const int m = r / CPH;
            const int c0 = grp * (NT / kEW) + (r - m * CPH) * kCHe;
            const int buf = it & 1;
            if (r == 0) {
                const uint32_t use = (uint32_t)(it >> 1);
                int go = 1;
                if (lane == 0)
                    go = WAITB(&phi_full[buf], use & 1u, 0x1000u) && WAITB(&tm_full[buf], use & 1u, 0x2000u);
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) return false;
                tc_fence_after();
            }
            // accumulator columns are read 8 at a time: fewer live registers than the whole chunk,
            // which keeps the several-problem loop (per-tile parameters in registers) from spilling
            constexpr int kY = 8;
            const uint32_t tcol = tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * (cpt / CPH) * NT + m * NT + c0);
            const int Qp = QP > 0 ? QP : t.Qp;
            const int ncell = t.ncell;
            const int fb = t.fb0 + c0;
            const int q = m * 128 + lq * 32 + lane;
            const bool live = fb < ncell && q < Qp;
            const bool pad = q >= t.Q;
            float* po = t.out + (size_t)(live ? fb : 0) * Qp + (live ? q : 0);
            const float4* cb = coef + buf * NT + c0;
            const float4 o4 = live ? __ldg(reinterpret_cast<const float4*>(t.ord) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float ax = fabsf(o4.x), ay = fabsf(o4.y), axy = ax + ay;
            const float dts = t.dts;
            const float ge = dts * o4.w;
            const int xbit = o4.x > 0.f ? 1 : (o4.x < 0.f ? 2 : 0);
#pragma unroll
            for (int h = 0; h < kCHe; h += kY) {
                float y[kY];
                __syncwarp();
                tmem_ld<kY>(tcol + (uint32_t)h, y);
                if (!live) continue;
#pragma unroll
                for (int j = 0; j < kY; ++j) {
                    const int i = h + j;
                    if (pad) {
                        if (fb + i < ncell) __stcs(po + i * Qp, 0.0f);
                        continue;
                    }
                    const float4 cf = cb[i];
                    const int bits = __float_as_int(cf.z);
                    if (!(bits & 16)) continue;
                    const float sf = s[i];
                    float upx = xbit == 1 ? (i > 0 ? s[i - 1] : lft) : (i < kCHe - 1 ? s[i + 1] : rgt);
                    upx = (bits & xbit) ? upx : 0.0f;
                    const float st = SPLIT ? sf : __bfloat162float(__float2bfloat16_rn(sf));
                    float out = fmaf(sf, cf.x - axy, cf.y);
                    out = fmaf(ax, upx, out);
                    out = fmaf(ay, u[i], out);
                    out = fmaf(dts, y[j], out);
                    out = fmaf(-ge, st, out);
                    __stcs(po + i * Qp, out);
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

        // Heun stage (the paper's explicit scheme, Sec. 3.1) of chunk r of a tile: kCHe cells;
        // x-stencil cells fb-2 .. fb+kCHe+1, y-rows two below / one below / one above (Omega_y > 0)
        // or one below / one above / two above (Omega_y < 0); out = alpha keep + beta (in + dt L(in)).
        auto heun_chunk = [&](const TileP& t, int it, int r, int cpt) -> bool {
            const int m = r / CPH;
            const int c0 = grp * (NT / kEW) + (r - m * CPH) * kCHe;
            const int ncell = t.ncell, nx = t.nx, Qp = QP > 0 ? QP : t.Qp;
            const int fb = t.fb0 + c0;
            const int q = m * 128 + lq * 32 + lane;
            const bool live = q < t.Q && fb < ncell;
            const float alpha = t.alpha, beta = t.beta;
            const float4 o4 = live ? __ldg(reinterpret_cast<const float4*>(t.ord) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
            const float nux = o4.x, nuy = o4.y;
            const float* b = t.in + (size_t)(live ? fb : 0) * Qp + (live ? q : 0);
            float sv[kCHe], ya[kCHe], yb[kCHe], yc[kCHe], kp[kCHe], e[4];
            // ya: row two below (nuy > 0) or two above (nuy < 0); yb: row below; yc: row above
            const long sy = (long)nx * Qp;
            const long da = nuy > 0.f ? -2 * sy : 2 * sy;
#pragma unroll
            for (int i = 0; i < kCHe; ++i) {
                const int f = fb + i;
                const bool in = live && f < ncell;
                sv[i] = in ? __ldg(b + i * Qp) : 0.0f;
                const bool ny0 = in && nuy != 0.f;
                ya[i] = (ny0 && (nuy > 0.f ? f >= 2 * nx : f + 2 * nx < ncell)) ? __ldg(b + i * Qp + da) : 0.0f;
                yb[i] = (ny0 && f >= nx) ? __ldg(b + i * Qp - sy) : 0.0f;
                yc[i] = (ny0 && f + nx < ncell) ? __ldg(b + i * Qp + sy) : 0.0f;
                kp[i] = (in && alpha != 0.0f) ? __ldg(t.keep + (size_t)f * Qp + q) : 0.0f;
            }
            e[0] = (live && fb >= 2) ? __ldg(b - 2 * Qp) : 0.0f;
            e[1] = (live && fb >= 1) ? __ldg(b - Qp) : 0.0f;
            e[2] = (live && fb + kCHe < ncell) ? __ldg(b + kCHe * Qp) : 0.0f;
            e[3] = (live && fb + kCHe + 1 < ncell) ? __ldg(b + (kCHe + 1) * Qp) : 0.0f;
            const int buf = it & 1;
            if (r == 0) {
                const uint32_t use = (uint32_t)(it >> 1);
                int go = 1;
                if (lane == 0)
                    go = WAITB(&phi_full[buf], use & 1u, 0x1000u) && WAITB(&tm_full[buf], use & 1u, 0x2000u);
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) return false;
                tc_fence_after();
            }
            float y[kCHe];
            __syncwarp();
            tmem_ld<kCHe>(tmem_base + ((uint32_t)(lq * 32) << 16) + (uint32_t)(buf * (cpt / CPH) * NT + m * NT + c0), y);
            if (fb < ncell && q < Qp) {
                float* po = t.out + (size_t)fb * Qp + q;
                const float4* cb = coef + buf * NT + c0;
                const float dts = t.dts, ge = dts * o4.w;
#pragma unroll
                for (int i = 0; i < kCHe; ++i) {
                    const float4 cf = cb[i];
                    const int bits = __float_as_int(cf.z);
                    if (!(bits & 16)) continue;
                    if (q >= t.Q) {
                        __stcs(po + i * Qp, 0.0f);
                        continue;
                    }
                    auto xv = [&](int k2) -> float { return k2 < 0 ? e[k2 + 2] : (k2 < kCHe ? sv[k2] : e[k2 - kCHe + 2]); };
                    const float xm2 = (bits & 32) ? xv(i - 2) : 0.0f;
                    const float xm1 = (bits & 1) ? xv(i - 1) : 0.0f;
                    const float xp1 = (bits & 2) ? xv(i + 1) : 0.0f;
                    const float xp2 = (bits & 64) ? xv(i + 2) : 0.0f;
                    const float c = sv[i];
                    const float tx = limited_difference(nux, xm2, xm1, c, xp1, xp2);
                    const bool up = nuy > 0.f;   // ya is two rows upwind: below for up, above otherwise
                    const float ty = limited_difference(nuy, up ? ya[i] : 0.0f, yb[i], c, yc[i], up ? 0.0f : ya[i]);
                    const float st = SPLIT ? c : __bfloat162float(__float2bfloat16_rn(c));
                    float adv = fmaf(c, cf.x, cf.y);
                    adv = fmaf(-nux, tx, adv);
                    adv = fmaf(-nuy, ty, adv);
                    adv = fmaf(dts, y[i], adv);
                    adv = fmaf(-ge, st, adv);
                    __stcs(po + i * Qp, fmaf(alpha, kp[i], beta * adv));
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
        // A chunk loaded and updated in one go (Heun, and the one-buffer forward-Euler form).
        float s0[kCHe], u0[kCHe], l0 = 0.f, r0 = 0.f;
        auto one_chunk = [&](const TileP& t, int it, int r, int cpt) -> bool {
            if constexpr (HEUN) {
                return heun_chunk(t, it, r, cpt);
            } else {
                load(t, r, s0, u0, l0, r0);
                return compute(t, it, r, cpt, s0, u0, l0, r0);
            }
        };

        if (a.one_fixed) {
            // One problem: its tiles blockIdx.x, blockIdx.x + gridDim.x, ... (all or none active);
            // chunk k of this warp is chunk k % cpt of the (k / cpt)-th of them.
            const int ntl = (s_info[0] & 2) ? total : 0;
            const int my_tiles = ntl > (int)blockIdx.x ? (ntl - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
            const int cpt = a.one.MB * CPH;
            const int nchunk = my_tiles * cpt;
            auto view = [&](int k, int& it, int& r) -> TileP {
                it = k / cpt;
                r = k - it * cpt;
                return TileP{a.one.in, a.one.out, a.one.ord, a.one.keep, ((int)blockIdx.x + it * (int)gridDim.x) * NT,
                             a.one.ncell, a.one.nx, a.one.Q, QP > 0 ? QP : a.one.Qp, a.one.dts, a.one.alpha, a.one.beta};
            };
            int it, r;
            if constexpr (kOneBuf) {
                for (int k = 0; k < nchunk && !*abort_flag; ++k) {
                    const TileP t = view(k, it, r);
                    if (!one_chunk(t, it, r, cpt)) break;
                }
            } else {
            float s1[kCHe], u1[kCHe], l1 = 0.f, r1 = 0.f;
            if (nchunk > 0) load(view(0, it, r), r, s0, u0, l0, r0);
            for (int k = 0; k < nchunk; k += 2) {
                if (k + 1 < nchunk) { const TileP t = view(k + 1, it, r); load(t, r, s1, u1, l1, r1); }
                { const TileP t = view(k, it, r); if (!compute(t, it, r, cpt, s0, u0, l0, r0)) break; }
                if (k + 1 >= nchunk) break;
                if (k + 2 < nchunk) { const TileP t = view(k + 2, it, r); load(t, r, s0, u0, l0, r0); }
                { const TileP t = view(k + 1, it, r); if (!compute(t, it, r, cpt, s1, u1, l1, r1)) break; }
            }
            }
        } else {
            // Several problems: walk the active tiles; the tile's parameters sit in this warp's
            // shared-memory slot (it & 1), rewritten from global memory only when the problem
            // changes (else copied from the other slot or kept).  A Heun launch takes each problem's
            // stage from its step counter: a Heun step is two launches and ends on the (even
            // distance) target, so the second stage runs when the counter's parity differs from the
            // target's; it keeps psi^n from the buffer it writes.
            struct Pos {
                int T, pid, it, r, cpt;
            };
            TileP* tslot = reinterpret_cast<TileP*>(base + L.tparm + e * 2 * 64);
            auto slot = [&](int it) -> const TileP& {
                return *reinterpret_cast<const TileP*>(reinterpret_cast<const unsigned char*>(tslot) + (it & 1) * 64);
            };
            int spid0 = -1, spid1 = -1;
            auto fill = [&](Pos& p) {
                if (p.T >= total) return;
                const int info = s_info[p.pid];
                p.cpt = ((info >> 16) & 255) * CPH;
                const int k = p.it & 1;
                TileP* t = reinterpret_cast<TileP*>(reinterpret_cast<unsigned char*>(tslot) + k * 64);
                const int mine = k ? spid1 : spid0, other = k ? spid0 : spid1;
                if (lane == 0) {
                    if (mine != p.pid) {
                        if (other == p.pid) {
                            *t = slot(p.it + 1);
                        } else {
                            const ProbDesc& d = a.probs[p.pid];
                            const int par = info & 1;
                            t->in = d.buf[par];
                            t->out = const_cast<float*>(d.buf[par ^ 1]);
                            t->ord = d.ord;
                            t->ncell = d.ncell;
                            t->nx = d.nx;
                            t->Q = d.Q;
                            t->Qp = QP > 0 ? QP : d.Qp;
                            t->dts = d.dt_sigma_as;
                            const bool stage2 = HEUN && ((par ^ d.target) & 1);
                            t->keep = stage2 ? t->out : nullptr;
                            t->alpha = stage2 ? 0.5f : 0.0f;
                            t->beta = stage2 ? 0.5f : 1.0f;
                        }
                    }
                    t->fb0 = (p.T - s_tile0[p.pid]) * NT;
                }
                if (k) spid1 = p.pid; else spid0 = p.pid;
                __syncwarp();
            };
            auto advance = [&](Pos& p) {
                if (++p.r < p.cpt) return;
                p.r = 0;
                ++p.it;
                p.T = next_tile(p.T + gridDim.x, p.pid);
                fill(p);
            };
            Pos cur;
            cur.it = 0;
            cur.r = 0;
            cur.pid = 0;
            cur.cpt = 1;
            cur.T = next_tile(blockIdx.x, cur.pid);
            fill(cur);
            if constexpr (kOneBuf) {
                while (cur.T < total && !*abort_flag) {
                    if (!one_chunk(slot(cur.it), cur.it, cur.r, cur.cpt)) break;
                    advance(cur);
                }
            } else {
            float s1[kCHe], u1[kCHe], l1 = 0.f, r1 = 0.f;
            if (cur.T < total) load(slot(cur.it), cur.r, s0, u0, l0, r0);
            while (cur.T < total) {
                Pos nxt = cur;
                advance(nxt);
                if (nxt.T < total) load(slot(nxt.it), nxt.r, s1, u1, l1, r1);
                if (!compute(slot(cur.it), cur.it, cur.r, cur.cpt, s0, u0, l0, r0)) break;
                cur = nxt;
                if (cur.T >= total) break;
                nxt = cur;
                advance(nxt);
                if (nxt.T < total) load(slot(nxt.it), nxt.r, s0, u0, l0, r0);
                if (!compute(slot(cur.it), cur.it, cur.r, cur.cpt, s1, u1, l1, r1)) break;
                cur = nxt;
            }
            }
        }
    }

    cp_async_wait<0>();   // converters: cell constants requested before an abort have landed
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tmem_base, 512);
    }
    // The last CTA to finish advances the step counters of the problems this launch stepped, unless
    // a bounded wait gave up (then no step is counted as taken).
    if (tid == 0) {
        __threadfence();
        const unsigned int done = atomicAdd(a.ticket, 1u);
        if (done == gridDim.x - 1) {
            __threadfence();
            const bool clean = *reinterpret_cast<volatile unsigned int*>(a.err) == 0u;
            for (int i = 0; i < nprob && clean; ++i)
                if (s_info[i] & 2) *a.probs[i].counter += 1;
            *a.ticket = 0u;
            __threadfence();
        }
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

// Flux buffer [ncell][Qp] FP32, box {64 ordinates, NT cells}, no swizzle.
bool encode_psi(CUtensorMap* map, const float* psi, int Qp, int ncell, int NT) {
    EncodeFn enc = get_encode();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)Qp, (cuuint64_t)ncell};
    const cuuint64_t strides[1] = {(cuuint64_t)Qp * 4};
    const cuuint32_t box[2] = {64, (cuuint32_t)NT};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(psi), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
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

size_t smem_for(int NT, bool split, int SS, int SB, int SA, int MPRmax) {
    auto need = [&](auto L) { return (size_t)1024 + (size_t)L.end; };
    switch (NT * 2 + (split ? 1 : 0)) {
        case 64: return need(Layout<32, false>(SS, SB, SA, MPRmax));
        case 65: return need(Layout<32, true>(SS, SB, SA, MPRmax));
        case 128: return need(Layout<64, false>(SS, SB, SA, MPRmax));
        case 129: return need(Layout<64, true>(SS, SB, SA, MPRmax));
        case 256: return need(Layout<128, false>(SS, SB, SA, MPRmax));
        case 257: return need(Layout<128, true>(SS, SB, SA, MPRmax));
        case 512: return need(Layout<256, false>(SS, SB, SA, MPRmax));
        default: return need(Layout<256, true>(SS, SB, SA, MPRmax));
    }
}

// Tile width, ring depths and request sizes for a set of problems.  Tile width: two accumulator
// buffers of MBmax x NT columns fill the 512 TMEM columns (or the requested width); narrower when
// the rings do not fit shared memory.  Rings: as requested (a zero field is chosen), else two
// staging and two operand stages and as many kernel-matrix stages of two ordinate blocks per
// request as fit (measured on the 448^2 / Q = 512 lattice: the kernel-matrix ring's depth in
// flight matters more than the other rings' and than fewer, larger requests).
bool choose_tiling(int MBmax, bool split, int want_nt, TcRings want, int& NT, int& SS, int& SB, int& SA,
                   int& MPRmax) {
    int nt = 512 / (2 * MBmax);
    if (nt > 256) nt = 256;
    if (want_nt) nt = want_nt;
    const size_t limit = 227 * 1024;
    while (true) {
        if (nt < 32 || (nt & (nt - 1)) || 2 * MBmax * nt > 512) return false;
        const int ss = want.SS ? want.SS : 2, sb = want.SB ? want.SB : 2;
        for (int mpr = want.MPR ? want.MPR : std::min(2, MBmax); mpr >= 1; mpr /= 2) {
            if (MBmax % mpr) continue;
            if (want.SA) {
                if (smem_for(nt, split, ss, sb, want.SA, mpr) <= limit) {
                    NT = nt; SS = ss; SB = sb; SA = want.SA; MPRmax = mpr;
                    return true;
                }
            } else if (smem_for(nt, split, ss, sb, 2, mpr) <= limit) {
                int sa = 2;
                while (sa < 8 && smem_for(nt, split, ss, sb, sa + 1, mpr) <= limit) ++sa;
                NT = nt; SS = ss; SB = sb; SA = sa; MPRmax = mpr;
                return true;
            }
            if (want.MPR) break;
        }
        if (want_nt) return false;
        nt /= 2;
    }
}

}  // namespace

struct Tc2Plan {
    int NT = 0, SS = 2, SB = 2, SA = 2, MPRmax = 1, QP = 0, grid = 0, total_tiles = 0, nprob = 0;
    bool split = false;
    size_t smem = 0;
    std::vector<ProbDesc> host;   // descriptors as uploaded
    ProbDesc* d_probs = nullptr;
    unsigned int* d_ticket = nullptr;
};

cudaError_t tc2_plan_create(Tc2Plan** out, const Tc2Problem* probs, int nprob, bool split, int want_nt,
                            TcRings rings) {
    *out = nullptr;
    if (nprob < 1 || nprob > kMaxProbs) return cudaErrorNotSupported;
    int MBmax = 1;
    for (int i = 0; i < nprob; ++i) MBmax = std::max(MBmax, probs[i].Mp / 128);
    Tc2Plan* p = new Tc2Plan();
    p->split = split;
    if (!choose_tiling(MBmax, split, want_nt, rings, p->NT, p->SS, p->SB, p->SA, p->MPRmax)) {
        delete p;
        return cudaErrorNotSupported;
    }
    p->smem = smem_for(p->NT, split, p->SS, p->SB, p->SA, p->MPRmax);
    p->nprob = nprob;
    p->host.resize(nprob);
    int tile0 = 0;
    for (int i = 0; i < nprob; ++i) {
        const Tc2Problem& s = probs[i];
        ProbDesc& d = p->host[i];
        memset(&d, 0, sizeof d);
        d.MB = s.Mp / 128;
        d.MPR = std::min(p->MPRmax, d.MB);
        while (d.MB % d.MPR) d.MPR /= 2;
        if (!encode_psi(&d.tm_psi[0], s.buf[0], s.Qp, s.nx * s.ny, p->NT) ||
            !encode_psi(&d.tm_psi[1], s.buf[1], s.Qp, s.nx * s.ny, p->NT) ||
            !encode_G4(&d.tm_hi, s.G_hi, s.Qp, d.MB, d.MPR) ||
            (split && !encode_G4(&d.tm_lo, s.G_lo, s.Qp, d.MB, d.MPR))) {
            delete p;
            return cudaErrorInvalidValue;
        }
        if (!split) d.tm_lo = d.tm_hi;
        d.buf[0] = s.buf[0];
        d.buf[1] = s.buf[1];
        d.ord = s.ord;
        d.cell = s.cell;
        d.w = s.w;
        d.counter = s.counter;
        d.target = s.target;
        d.nx = s.nx;
        d.ny = s.ny;
        d.ncell = s.nx * s.ny;
        d.Q = s.Q;
        d.Qp = s.Qp;
        d.KC = s.Qp / 64;
        d.ntiles = (d.ncell + p->NT - 1) / p->NT;
        d.tile0 = tile0;
        d.dt = s.dt;
        d.dt_sigma_as = s.dt_sigma_as;
        tile0 += d.ntiles;
    }
    p->total_tiles = tile0;
    // compile-time stride when every problem shares one ordinate stride
    p->QP = probs[0].Qp;
    for (int i = 1; i < nprob; ++i)
        if (probs[i].Qp != p->QP) p->QP = 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    p->grid = std::min(p->total_tiles, sms);
    cudaError_t e = cudaMalloc(&p->d_probs, sizeof(ProbDesc) * nprob);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_ticket, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(p->d_ticket, 0, sizeof(unsigned int));
    if (e == cudaSuccess)
        e = cudaMemcpy(p->d_probs, p->host.data(), sizeof(ProbDesc) * nprob, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        tc2_plan_destroy(p);
        return e;
    }
    *out = p;
    return cudaSuccess;
}

void tc2_plan_destroy(Tc2Plan* p) {
    if (!p) return;
    if (p->d_probs) cudaFree(p->d_probs);
    if (p->d_ticket) cudaFree(p->d_ticket);
    delete p;
}

void tc2_plan_describe(const Tc2Plan* p, int* tile_cells, int* stages, int* tmem_cols, size_t* smem) {
    if (tile_cells) *tile_cells = p ? p->NT : 0;
    if (stages) *stages = p ? p->SA : 0;
    if (tmem_cols) *tmem_cols = p ? 512 : 0;
    if (smem) *smem = p ? p->smem : 0;
}

int tc2_plan_total_tiles(const Tc2Plan* p) { return p ? p->total_tiles : 0; }

TcRings tc2_plan_rings(const Tc2Plan* p) {
    TcRings r;
    if (p) {
        r.SS = p->SS;
        r.SB = p->SB;
        r.SA = p->SA;
        r.MPR = p->MPRmax;
    }
    return r;
}

cudaError_t tc2_plan_set_targets(Tc2Plan* p, const int* targets, cudaStream_t stream) {
    if (!p) return cudaErrorInvalidValue;
    bool changed = false;
    for (int i = 0; i < p->nprob; ++i) {
        if (p->host[i].target != targets[i]) changed = true;
        p->host[i].target = targets[i];
    }
    if (!changed) return cudaSuccess;
    // the host table outlives the copy (pageable source: staged before the call returns)
    return cudaMemcpyAsync(p->d_probs, p->host.data(), sizeof(ProbDesc) * p->nprob, cudaMemcpyHostToDevice, stream);
}

template <int NT, bool SPLIT, int QP, bool HEUN = false>
static cudaError_t launch2(const Tc2Plan* p, const BatchArgs& a, cudaStream_t s) {
    auto kern = step_tc2_kernel<NT, SPLIT, QP, HEUN>;
    cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    if (r != cudaSuccess) return r;
    kern<<<p->grid, Roles<NT, SPLIT, QP, HEUN>::kThreads, p->smem, s>>>(a);
    return cudaGetLastError();
}

// Compile-time ordinate strides for the common quadratures (at their automatic tile widths and
// half of them); everything else runs the runtime-stride instance.
template <bool SPLIT>
static cudaError_t dispatch(const Tc2Plan* p, const BatchArgs& a, cudaStream_t s) {
    const int key = p->QP * 1000 + p->NT;
    switch (key) {
        case 512 * 1000 + 64: return launch2<64, SPLIT, 512>(p, a, s);
        case 512 * 1000 + 32: return launch2<32, SPLIT, 512>(p, a, s);
        case 256 * 1000 + 128: return launch2<128, SPLIT, 256>(p, a, s);
        case 256 * 1000 + 64: return launch2<64, SPLIT, 256>(p, a, s);
        case 128 * 1000 + 256: return launch2<256, SPLIT, 128>(p, a, s);
        case 128 * 1000 + 128: return launch2<128, SPLIT, 128>(p, a, s);
        case 64 * 1000 + 256: return launch2<256, SPLIT, 64>(p, a, s);
        case 64 * 1000 + 128: return launch2<128, SPLIT, 64>(p, a, s);
        default: break;
    }
    switch (p->NT) {
        case 32: return launch2<32, SPLIT, 0>(p, a, s);
        case 64: return launch2<64, SPLIT, 0>(p, a, s);
        case 128: return launch2<128, SPLIT, 0>(p, a, s);
        default: return launch2<256, SPLIT, 0>(p, a, s);
    }
}

template <bool SPLIT>
static cudaError_t dispatch_heun(const Tc2Plan* p, const BatchArgs& a, cudaStream_t s) {
    switch (p->NT) {
        case 32: return launch2<32, SPLIT, 0, true>(p, a, s);
        case 64: return launch2<64, SPLIT, 0, true>(p, a, s);
        case 128: return launch2<128, SPLIT, 0, true>(p, a, s);
        default: return launch2<256, SPLIT, 0, true>(p, a, s);
    }
}

static BatchArgs batch_args(Tc2Plan* p, unsigned int* err_flag, int parity0);

cudaError_t launch_heun_stage_tc2(Tc2Plan* p, unsigned int* err_flag, int parity0, const float* keep, float alpha,
                                  float beta, cudaStream_t stream) {
    if (!p || (parity0 >= 0 && p->nprob != 1)) return cudaErrorInvalidValue;
    BatchArgs a = batch_args(p, err_flag, parity0);
    a.one.keep = keep;
    a.one.alpha = alpha;
    a.one.beta = beta;
    return p->split ? dispatch_heun<true>(p, a, stream) : dispatch_heun<false>(p, a, stream);
}

cudaError_t launch_step_tc2(Tc2Plan* p, unsigned int* err_flag, int parity0, cudaStream_t stream) {
    if (!p) return cudaErrorInvalidValue;
    const BatchArgs a = batch_args(p, err_flag, parity0);
    return p->split ? dispatch<true>(p, a, stream) : dispatch<false>(p, a, stream);
}

static BatchArgs batch_args(Tc2Plan* p, unsigned int* err_flag, int parity0) {
    BatchArgs a;
    for (int i = 0; i < kParamProbs && i < p->nprob; ++i) {
        const ProbDesc& d = p->host[i];
        a.pm[i].psi[0] = d.tm_psi[0];
        a.pm[i].psi[1] = d.tm_psi[1];
        a.pm[i].hi = d.tm_hi;
        a.pm[i].lo = d.tm_lo;
    }
    a.one_fixed = (p->nprob == 1 && parity0 >= 0) ? 1 : 0;
    {
        const ProbDesc& d = p->host[0];
        a.one.in = d.buf[parity0 & 1];
        a.one.out = const_cast<float*>(d.buf[(parity0 & 1) ^ 1]);
        a.one.ord = d.ord;
        a.one.ncell = d.ncell;
        a.one.nx = d.nx;
        a.one.Q = d.Q;
        a.one.Qp = d.Qp;
        a.one.MB = d.MB;
        a.one.dts = d.dt_sigma_as;
    }
    a.probs = p->d_probs;
    a.nprob = p->nprob;
    a.total_tiles = p->total_tiles;
    a.err = err_flag;
    a.ticket = p->d_ticket;
    a.SS = p->SS;
    a.SB = p->SB;
    a.SA = p->SA;
    a.MPRmax = p->MPRmax;
    a.one.keep = nullptr;
    a.one.alpha = 0.0f;
    a.one.beta = 1.0f;
    return a;
}

}  // namespace assn
