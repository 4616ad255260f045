// Paired-SM tensor-core as-S_N step (sm_103a): one problem, forward Euler with first-order upwind
// transport (Sec. 3.1-3.2), 256 or 512 ordinates (padded), FP32 state; the contraction in BF16, in
// BF16X3 (both operands split), in BF16X2 (the kernel matrix split, the operand in one BF16 part) or
// in TF32.
//
// A cluster of two CTAs on two SMs (the pair) steps one tile of TW x TH cells per round (TW = 16;
// TH = 8 at 512 ordinates, 16 at 256; tiles row-major over the grid, pair p takes tiles p, p + P, ...).
// The artificial in-scattering gain without its diagonal (Sec. 3.2, Eq. (as-S_N equations))
//   D[q][c] = sum_{p != q} G_qp psi~_p(c)
// is computed by tcgen05.mma.cta_group::2 products of M = 256 ordinates x N = TW TH cells x K = 16
// (BF16 in, FP32 accumulate in tensor memory; K = 8 in TF32, whose 64-ordinate chunk is two
// 32-ordinate halves of 128-byte rows, laid out like the hi and lo parts of the split contraction).
// In each 256-ordinate group the even CTA holds
// rows 0-127 of G and of the accumulator, the odd CTA rows 128-255; each CTA converts and holds
// the operand rows of half the tile's cells (rows 0 .. TH/2-1 in the even CTA).  Each SM thus
// loads half of G per tile and supplies half the operand bytes of every MMA.
//
// Roles in each CTA (20 warps: 96 registers per thread):
//   warp 0      TMEM (both CTAs allocate the pair's 512 columns collectively); lane 0 of the even
//               CTA issues the MMAs into one of two accumulator buffers and commits to the
//               barriers of both CTAs; lane 0 of the odd CTA forwards the completion of its own
//               kernel-matrix copies to the even CTA.
//               Lane 2: TMA of this CTA's G rows ([128 x 64] BF16 blocks, or [128 x 32] TF32 ones,
//               with 128-byte swizzle): its distinct BF16 blocks once (resident), or all of its
//               256-row groups, one or two chunks per request, through a ring.
//   flux TMA    this CTA's half tile of FP32 flux, [TW x TH/2 cells x 64 ordinates] chunks, into a
//               staging ring: warp 3 at 512 ordinates, else lane 1 of warp 0.
//   warps 1-3   converters (1-2 at 512 ordinates): staging -> BF16 (hi [+ lo]) or TF32 operand
//               rows (K-major, swizzled) for the pair's MMA;
//               the scalar flux Phi = sum_p w_p psi_p of this CTA's cells, and from it the cells'
//               coefficients, written into both CTAs.
//   warps 4-19  epilogue: warp (lane quarter lq, group g) owns 32 ordinates of one 128-row block
//               and an 8-cell-wide strip of the tile, and walks its 8 rows in order; the upwind
//               y-neighbour is the previous or next row of the walk (in registers), the upwind
//               x-neighbour the next register or one edge cell per row:
//                 psi' = psi (1 - dt sigma_t - a_x - a_y) + a_x psi_upx + a_y psi_upy
//                        + dt (sigma_s Phi / sum w + q) + dt sigma_as (D - e psi~)
//               Tiles away from the boundary take a branch-free path (pairs of cells per FFMA2).
//
// Every wait is bounded (about 1 s); on expiry the CTA records the event in err, stops issuing,
// lets its own copies and MMAs land (bounded again), and both CTAs meet at the final cluster
// barrier before the tensor memory is freed.
#include <string.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "assn_internal.h"
#include "tc_ptx.h"

namespace assn {

namespace {

using namespace ptx;

constexpr int kTW = 16;                 // tile width (cells)
constexpr int kEpi3 = 16;               // epilogue warps (4 .. 19; any four consecutive warps cover the
                                        // four TMEM lane quarters, warp & 3)
constexpr int kEpi0 = 4;                // first epilogue warp; warps 1-3 convert, or 1-2 convert and 3
                                        // requests the flux copies
constexpr int kThreads3 = (kEpi0 + kEpi3) * 32;
constexpr int kABlock = 128 * 64 * 2;   // one [128 x 64] BF16 block of G

struct Tc3Args {
    CUtensorMap tm_psi;                 // input flux [ny][nx][Qp] FP32, box {64, TW, TH/2}
    CUtensorMap tm_G;                   // G [Mp][Qp] BF16 as {64, 128, 2, MG, KC}, box {64, 128, 1, MG, CPS}
                                        // (TF32: {32, 128, 2, MG, 2 KC}, box {32, 128, 1, MG, 1})
    CUtensorMap tm_Glo;                 // split contraction: the residual of G, same view
    const float* in;
    float* out;
    const OrdF* ord;                    // [Qp]
    const CellF* cell;                  // [ncell]
    const float* w;                     // [Qp]
    unsigned int* err;
    // resident kernel matrix (nslot > 0): the distinct [128 x 64] blocks of this CTA's rows, loaded
    // once; 4-bit fields indexed by kc MG + j (chunk kc, group j): slots = the slot holding that
    // block, reps = for slot s, the index kc MG + j it is loaded from
    unsigned long long slots, reps;
    int nslot;
    int nx, ny, Q, ntx, total;
    int SS, SB, SA;
    float dt, dts;                      // dt and dt sigma_as
    // Heun stage (HEUN instances): out = alpha keep + beta (in + dt L(in)); keep may be out itself
    const float* keep;
    float alpha, beta;
};

// Contraction precision of a kernel instance: one BF16 pass, the BF16X3 split, one TF32 pass, or
// BF16X2 (G hi x psi~ + G lo x psi~).
constexpr int kPrBF16 = 0, kPrSplit = 1, kPrTF32 = 2, kPrX2 = 3;

template <int MG, int CPS_ = 2, int PR = kPrBF16>
struct L3 {
    static constexpr int NT = 256 / MG;         // cells per tile (MMA N)
    static constexpr int TH = NT / kTW;         // tile rows
    static constexpr int THc = TH / 2;          // rows per CTA
    static constexpr int NTc = NT / 2;          // cells per CTA
    static constexpr int QP = 256 * MG;         // ordinate stride
    static constexpr int KC = QP / 64;          // 64-ordinate chunks
    static constexpr int CPS = CPS_;            // chunks per operand / kernel-matrix stage (one MMA round)
    static constexpr int KR = KC / CPS;         // MMA rounds per tile
    static constexpr int kStg = NTc * 256;      // FP32 staging stage (one chunk)
    // parts of a chunk: hi [+ lo] BF16, or the two 32-ordinate halves of a TF32 chunk (each part
    // [rows x 128 B], so a TF32 stage has the split contraction's layout); BF16X2 splits G only
    static constexpr int NPA = PR == kPrBF16 ? 1 : 2;                   // kernel-matrix parts
    static constexpr int NPB = PR == kPrBF16 || PR == kPrX2 ? 1 : 2;    // operand parts
    static constexpr int kB = NPB * CPS * NTc * 128;     // operand stage (first parts of the CPS chunks, then second)
    static constexpr int kA = NPA * CPS * MG * kABlock;  // G stage: this CTA's blocks of CPS chunks (first parts, then second)
    int stg, b, a, cx, cy, cb, cst, wsm, bars, end;
    __host__ __device__ L3(int SS, int SB, int SA, int nslot) {
        stg = 0;
        b = stg + SS * kStg;
        a = b + SB * kB;
        // kernel matrix: nslot resident blocks, else a ring of SB stages (the operand ring's depth)
        cx = a + (nslot > 0 ? nslot * kABlock : SB * kA);   // [2][NT] 1 - dt sigma_t
        cy = cx + 2 * NT * 4;                   // [2][NT] dt (sigma_s Phi / sum w + q)
        cb = cy + 2 * NT * 4;                   // [2][NT] neighbour bits
        cst = cb + 2 * NT * 4;                  // [NTc] cell constants of this CTA's cells
        wsm = cst + NTc * 16;                   // [QP] quadrature weights
        bars = wsm + QP * 4;
        // stg full/empty [SS], stage full/pair/empty [SB] (operand and kernel-matrix rings advance
        // together, SA == SB), tm full/empty [2], phi full/empty [2], drain, resident kernel matrix
        end = bars + 8 * (2 * SS + 3 * SB + 10) + 16;
    }
};

struct Ring3 {
    int s = 0;
    uint32_t ph = 0;
    __device__ __forceinline__ void next(int S) {
        if (++s == S) { s = 0; ph ^= 1u; }
    }
};

// Local-scope and cluster-scope bounded waits, fast path inline.
#define W3(bar, parity, code) (mbar_try_wait((bar), (parity)) || mbar_wait((bar), (parity), abort_flag, a.err, (code)))
#define W3C(bar, parity, code) \
    (mbar_try_wait_cl((bar), (parity)) || mbar_wait_cl((bar), (parity), abort_flag, a.err, (code)))


__device__ __forceinline__ float bf16_round(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// minmod of two one-sided differences: the one of smaller magnitude when they agree in sign, else 0
__device__ __forceinline__ float minmod3(float a, float b) {
    return a * b > 0.0f ? (fabsf(a) < fabsf(b) ? a : b) : 0.0f;
}

// psi~ as the contraction sees it: rounded to BF16 (BF16, BF16X2), itself (split: hi + lo carry it to
// about 2^-16), or rounded to TF32
template <int PR>
__device__ __forceinline__ float operand_value(float v) {
    if constexpr (PR == kPrBF16 || PR == kPrX2) return bf16_round(v);
    else if constexpr (PR == kPrTF32) return tf32_round(v);
    else return v;
}

// HEUN: one stage of Heun's method with minmod-limited second-order upwind fluxes (Sec. 3.1):
// out = alpha keep + beta (in + dt L(in)), L with the limited transport, collision, scattering,
// source and the artificial gain of the stage state.
template <int MG, int CPS_, int PR, bool HEUN = false>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads3, 1)
step_tc3_kernel(const __grid_constant__ Tc3Args a) {
    using LT = L3<MG, CPS_, PR>;
    constexpr bool SPLIT = PR == kPrSplit, TF = PR == kPrTF32, X2 = PR == kPrX2;
    // converter warps and where the flux-copy producer runs: at 512 ordinates (16-kB chunks) two
    // converter warps keep up and the producer gets warp 3 to itself (as one lane of warp 0, beside
    // the MMA issuer's waits, it issued each copy about a microsecond after its slot was released:
    // on the 448^2 lattice 0.180 -> 0.174 ms in BF16, 0.334 -> 0.288 ms in BF16X3); the 32-kB chunks
    // at 256 ordinates need three converter warps (2.14 against 1.80-1.95 ms on the 2048^2 line source)
    constexpr int kConv3 = MG == 2 ? 2 : 3;
    constexpr bool kProdWarp = kConv3 == 2;
    constexpr int NT = LT::NT, TH = LT::TH, THc = LT::THc, NTc = LT::NTc, QP = LT::QP, KC = LT::KC;
    constexpr int CPS = LT::CPS, KR = LT::KR;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    const LT L(a.SS, a.SB, a.SA, a.nslot);
    const bool resident = a.nslot > 0;
    float* stg = reinterpret_cast<float*>(base + L.stg);
    unsigned char* bring = base + L.b;
    unsigned char* aring = base + L.a;
    float* cx = reinterpret_cast<float*>(base + L.cx);
    float* cy = reinterpret_cast<float*>(base + L.cy);
    int* cb = reinterpret_cast<int*>(base + L.cb);
    CellF* cst = reinterpret_cast<CellF*>(base + L.cst);
    float4* wsm = reinterpret_cast<float4*>(base + L.wsm);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + L.bars);
    uint64_t* stg_full = bars;
    uint64_t* stg_empty = stg_full + a.SS;
    // one stage of the operand ring and of the kernel-matrix ring share a barrier set: full
    // (this CTA's converter warps arrive, the kernel-matrix copy completes its bytes), pair (the odd
    // CTA's full, forwarded to the even CTA), empty (the pair's MMAs of the stage completed)
    uint64_t* st_full = stg_empty + a.SS;
    uint64_t* st_pair = st_full + a.SB;
    uint64_t* st_empty = st_pair + a.SB;
    uint64_t* tm_full = st_empty + a.SB;
    uint64_t* tm_empty = tm_full + 2;
    uint64_t* phi_full = tm_empty + 2;
    uint64_t* phi_empty = phi_full + 2;
    uint64_t* drain_bar = phi_empty + 2;
    uint64_t* gres = drain_bar + 1;      // the resident kernel-matrix blocks have landed
    uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(gres + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t rank = cluster_ctarank();
    const int pair = blockIdx.x >> 1, npair = gridDim.x >> 1;
    const int total = a.total;

    if (tid == 0) {
        for (int s = 0; s < a.SS; ++s) { mbar_init(&stg_full[s], 1); mbar_init(&stg_empty[s], kConv3); }
        for (int s = 0; s < a.SB; ++s) {
            mbar_init(&st_full[s], kConv3 + (resident ? 0 : 1));   // + the kernel-matrix copy when streamed
            mbar_init(&st_pair[s], 1);
            mbar_init(&st_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tm_full[b], 1);
            mbar_init(&tm_empty[b], 2 * kEpi3);
            mbar_init(&phi_full[b], kConv3);   // + the peer's coefficient bytes (st.async)
            mbar_init(&phi_empty[b], 2 * kEpi3);
        }
        mbar_init(drain_bar, 1);
        mbar_init(gres, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    for (int i = tid; i < QP / 4; i += blockDim.x) wsm[i] = __ldg(reinterpret_cast<const float4*>(a.w) + i);
    if (warp == 0) {
        tmem_alloc_pair(tmem_holder, 512);
        tc_fence_before();
    }
    __syncthreads();
    cluster_sync();   // the peer's barriers are initialised and its tensor memory allocated
    tc_fence_after();
    const uint32_t tmem_base = *tmem_holder;

    // flux TMA producer: this CTA's half tile of FP32 flux, [TW x TH/2 cells x 64 ordinates]
    // chunks, into the staging ring
    auto flux_producer = [&]() {
        const uint64_t pol = policy_evict_last();   // the epilogue re-reads these lines shortly
        Ring3 rs;
        uint32_t armed = 0u, apar = 0u;
        for (int T = pair; T < total; T += npair) {
            const int ty = T / a.ntx, tx = T - ty * a.ntx;
            bool ok = true;
            for (int kc = 0; kc < KC; ++kc) {
                if (!W3(&stg_empty[rs.s], rs.ph ^ 1u, 0x1u)) { ok = false; break; }
                mbar_expect_tx(&stg_full[rs.s], LT::kStg);
                tma_load_3d_hint(stg + (size_t)rs.s * NTc * 64, &a.tm_psi, &stg_full[rs.s], kc * 64, tx * kTW,
                                 ty * TH + (int)rank * THc, pol);
                armed |= 1u << rs.s;
                apar = (apar & ~(1u << rs.s)) | (rs.ph << rs.s);
                rs.next(a.SS);
            }
            if (!ok) break;
        }
        if (*abort_flag)
            for (int s2 = 0; s2 < a.SS; ++s2)
                if (((armed >> s2) & 1u) && !mbar_drain(&stg_full[s2], (apar >> s2) & 1u, kDrainNs))
                    atomicOr(a.err, kErrUndrained);
    };

    if (warp == 0) {
        if (lane == 0 && rank == 0) {
            // ------------------------------------------------------------------------ MMA issuer
            constexpr uint32_t idesc = TF ? idesc_tf32(256, NT) : idesc_bf16(256, NT);
            const uint64_t a0 = sw128_desc(smem_u32(aring));
            const uint64_t b0 = sw128_desc(smem_u32(bring));
            Ring3 rq;
            bool ok = !resident || W3(gres, 0u, 0x80u);
            tc_fence_after();
            for (int T = pair, it = 0; T < total && ok; T += npair, ++it) {
                const int buf = it & 1;
                const uint32_t use = (uint32_t)(it >> 1);
                if (!W3(&tm_empty[buf], (use & 1u) ^ 1u, 0x10u)) break;
                tc_fence_after();
                const uint32_t dbase = tmem_base + (uint32_t)(buf * MG * NT);
                for (int kr = 0; kr < KR; ++kr) {
                    if (!W3(&st_full[rq.s], rq.ph, 0x20u) || !W3(&st_pair[rq.s], rq.ph, 0x40u)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t bd0 = b0 + (uint64_t)((rq.s * LT::kB) >> 4);
                    const uint64_t ad0 = a0 + (uint64_t)((rq.s * LT::kA) >> 4);
#pragma unroll
                    for (int c = 0; c < CPS; ++c) {
#pragma unroll
                        for (int j = 0; j < MG; ++j) {
                            // this round's block of group j: its resident slot, else its place in the stage
                            const int blk = resident ? (int)((a.slots >> (4 * ((kr * CPS + c) * MG + j))) & 15u)
                                                     : c * MG + j;
                            const uint64_t ab = resident ? a0 : ad0;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ah = ab + (uint64_t)((blk * kABlock) >> 4) + (uint64_t)(kk * 2);
                                const uint64_t bh = bd0 + (uint64_t)((c * NTc * 128) >> 4) + (uint64_t)(kk * 2);
                                const uint32_t dd = dbase + (uint32_t)(j * NT);
                                // (second parts of the stage: the lo parts, or the TF32 chunks' upper halves)
                                const uint64_t bh2 = bh + (uint64_t)((CPS * NTc * 128) >> 4);
                                const uint64_t ah2 = ah + (uint64_t)((CPS * MG * kABlock) >> 4);
                                if constexpr (TF) {   // ordinates 8 kk .. + 7 of each 32-ordinate half
                                    mma_tf32_pair(dd, ah, bh, idesc, (kr > 0 || c > 0 || kk > 0) ? 1u : 0u);
                                    mma_tf32_pair(dd, ah2, bh2, idesc, 1u);
                                } else {
                                    mma_bf16_pair(dd, ah, bh, idesc, (kr > 0 || c > 0 || kk > 0) ? 1u : 0u);
                                    if (SPLIT) {   // + hi x lo + lo x hi (the lo parts follow the CPS hi chunks)
                                        mma_bf16_pair(dd, ah, bh2, idesc, 1u);
                                        mma_bf16_pair(dd, ah2, bh, idesc, 1u);
                                    }
                                    if (X2) mma_bf16_pair(dd, ah2, bh, idesc, 1u);   // + G lo x psi~
                                }
                            }
                        }
                    }
                    mma_commit_pair(&st_empty[rq.s], 3);
                    rq.next(a.SB);
                }
                mma_commit_pair(&tm_full[buf], 3);
            }
            if (*abort_flag) {   // every MMA issued completes before the pair's tensor memory is freed
                mma_commit_pair(drain_bar, 1);
                if (!mbar_drain(drain_bar, 0u, kDrainNs)) atomicOr(a.err, kErrUndrained);
            }
        } else if (lane == 0) {
            // ------------------------- odd CTA: forward its operand and kernel-matrix completions
            // (the converters and the TMA signal this CTA's barriers; the data is complete in this
            // CTA's shared memory when they do, and this thread republishes each completion to the
            // even CTA, whose MMAs then read it)
            const uint32_t pair0 = mapa_shared(smem_u32(st_pair), 0);
            Ring3 rq;
            // (with a resident kernel matrix, the first completion forwarded also vouches for its blocks)
            const bool res_ok = !resident || W3(gres, 0u, 0x4000u);
            for (int T = pair; T < total && res_ok; T += npair) {
                bool ok = true;
                for (int kr = 0; kr < KR; ++kr) {
                    if (!W3(&st_full[rq.s], rq.ph, 0x400u)) { ok = false; break; }
                    mbar_arrive_remote(pair0 + 8u * (uint32_t)rq.s);
                    rq.next(a.SB);
                }
                if (!ok) break;
            }
        } else if (lane == 1) {
            if (!kProdWarp) flux_producer();
        } else if (lane == 2) {
            // --------------------------------------------------------- kernel-matrix TMA producer
            const uint64_t pol = policy_evict_last();   // every tile re-reads G from L2
            Ring3 rq;
            uint32_t armed = 0u, apar = 0u;
            if (resident) {
                // the distinct blocks of this CTA's rows, once; this thread waits (bounded) for them
                // to land so that no copy is in flight at teardown, whatever the other roles do
                mbar_expect_tx(gres, (uint32_t)(a.nslot * kABlock));
                for (int sl = 0; sl < a.nslot; ++sl) {
                    const int idx = (int)((a.reps >> (4 * sl)) & 15u);
                    tma_load_5d_hint(aring + (size_t)sl * kABlock, &a.tm_G, gres, 0, 0, (int)rank, idx % MG, idx / MG,
                                     pol);
                }
                if (!mbar_drain(gres, 0u, kDrainNs)) atomicOr(a.err, kErrUndrained);
            }
            for (int T = pair; T < total && !resident; T += npair) {
                bool ok = true;
                for (int kr = 0; kr < KR; ++kr) {
                    if (!W3(&st_empty[rq.s], rq.ph ^ 1u, 0x2u)) { ok = false; break; }
                    mbar_expect_tx(&st_full[rq.s], LT::kA);
                    // TF32: G's 32-column chunks 2 kr and 2 kr + 1 (one 64-ordinate chunk per stage)
                    const int gch = TF ? 2 * kr : kr * CPS;
                    tma_load_5d_hint(aring + (size_t)rq.s * LT::kA, &a.tm_G, &st_full[rq.s], 0, 0, (int)rank, 0, gch,
                                     pol);
                    if (SPLIT || TF || X2)
                        tma_load_5d_hint(aring + (size_t)rq.s * LT::kA + LT::kA / 2, TF ? &a.tm_G : &a.tm_Glo,
                                         &st_full[rq.s], 0, 0, (int)rank, 0, TF ? gch + 1 : gch, pol);
                    armed |= 1u << rq.s;
                    apar = (apar & ~(1u << rq.s)) | (rq.ph << rq.s);
                    rq.next(a.SB);
                }
                if (!ok) break;
            }
            if (*abort_flag)   // (the stage's phase also waits for the converters, which stop on abort)
                for (int s2 = 0; s2 < a.SB; ++s2)
                    if (((armed >> s2) & 1u) && !mbar_drain(&st_full[s2], (apar >> s2) & 1u, kDrainNs))
                        atomicOr(a.err, kErrUndrained);
        }
    } else if (kProdWarp && warp == 1 + kConv3) {
        if (lane == 0) flux_producer();
    } else if (warp <= kConv3) {
        // ------------------------------------------------------------------------ converters
        // Thread (rsub, col4) converts float4 column col4 of the cells rsub, rsub + RS, ... of each
        // staged chunk and owns the cell constants and coefficients of cells col4 + 16 k of its
        // column (when there are that many).  No global memory is read inside the chunk loop
        // (weights in shared memory, cell constants requested at the start of the tile).
        constexpr int RS = 2 * kConv3;       // rows (cells) advanced per step of a thread column
        constexpr int NR = (NTc + RS - 1) / RS;   // cells per thread (the last step is partial)
        constexpr int NOWN = (NR + 15) / 16; // cells whose coefficients this thread may write
        const int ct = tid - 32;             // 0 .. 32 kConv3 - 1
        const int rsub = ct >> 4;
        const int col4 = ct & 15;
        const uint32_t phi_rem = mapa_shared(smem_u32(phi_full), rank ^ 1u);
        const uint32_t cx_rem = mapa_shared(smem_u32(cx), rank ^ 1u);
        const uint32_t cy_rem = mapa_shared(smem_u32(cy), rank ^ 1u);
        const uint32_t cb_rem = mapa_shared(smem_u32(cb), rank ^ 1u);
        const float dt = a.dt;
        // byte offset of this thread's operand store for row r (float4 column col4, canonical
        // K-major layout with 128-byte swizzle: BF16, 8 bytes in 16-byte unit col4 / 2 of the row;
        // TF32, the 16-byte unit col4 % 8 of the row in half col4 / 8); fixed for the whole launch,
        // so kept in registers where a thread has few rows
        auto store_off = [col4](int r) {
            if constexpr (TF)
                return (col4 >> 3) * (CPS * NTc * 128) + (r >> 3) * 1024 + (r & 7) * 128 + (((col4 & 7) ^ (r & 7)) << 4);
            else
                return (r >> 3) * 1024 + (r & 7) * 128 + (((col4 >> 1) ^ (r & 7)) << 4) + ((col4 & 1) << 3);
        };
        constexpr bool kKeepOffs = NR <= 11;
        int offs[kKeepOffs ? NR : 1];
#pragma unroll
        for (int i = 0; i < (kKeepOffs ? NR : 1); ++i) offs[i] = store_off(rsub + RS * i);
        Ring3 rs, rb;
        for (int T = pair, it = 0; T < total; T += npair, ++it) {
            const int ty = T / a.ntx, tx = T - ty * a.ntx;
            const int xbase = tx * kTW, ybase = ty * TH + (int)rank * THc;
#pragma unroll
            for (int k = 0; k < NOWN; ++k) {
                const int i = col4 + 16 * k;
                const int r = rsub + RS * i;
                const int xx = xbase + (r & (kTW - 1)), yy = ybase + r / kTW;
                if (i < NR && r < NTc && xx < a.nx && yy < a.ny)
                    cp_async16(smem_u32(cst + r), a.cell + (size_t)yy * a.nx + xx, 16u);
            }
            cp_async_commit();
            float part[NR];
#pragma unroll
            for (int i = 0; i < NR; ++i) part[i] = 0.0f;
            bool ok = true;
            for (int kc = 0; kc < KC; ++kc) {
                const int sub = kc % CPS;    // chunk within the operand stage
                if (!W3(&stg_full[rs.s], rs.ph, 0x100u) || (sub == 0 && !W3(&st_empty[rb.s], rb.ph ^ 1u, 0x200u))) {
                    ok = false;
                    break;
                }
                const float4 w4 = wsm[kc * 16 + col4];
                const float4* src = reinterpret_cast<const float4*>(stg + (size_t)rs.s * NTc * 64);
                unsigned char* dst = bring + rb.s * LT::kB + sub * NTc * 128;
                const float2 wa = make_float2(w4.x, w4.y), wb = make_float2(w4.z, w4.w);
                // groups of up to GR rows: all shared-memory loads of a group first, then the
                // arithmetic and the operand stores (the rows are independent, so the loads overlap)
                constexpr int GR = NR <= 11 ? NR : 8;      // (22 rows at 256 ordinates: groups of 8)
#pragma unroll
                for (int i0 = 0; i0 < NR; i0 += GR) {
                    float4 v[GR];
#pragma unroll
                    for (int g = 0; g < GR; ++g) {
                        const int r = rsub + RS * (i0 + g);
                        v[g] = (i0 + g < NR && r < NTc) ? src[r * 16 + col4] : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
#pragma unroll
                    for (int g = 0; g < GR; ++g) {
                        const int i = i0 + g;
                        const int r = rsub + RS * i;
                        if (i >= NR || r >= NTc) continue;
                        const float2 pp = __ffma2_rn(wb, make_float2(v[g].z, v[g].w), __fmul2_rn(wa, make_float2(v[g].x, v[g].y)));
                        part[i] += pp.x + pp.y;
                        const int off = kKeepOffs ? offs[kKeepOffs ? i : 0] : store_off(r);
                        if constexpr (TF) {
                            *reinterpret_cast<uint4*>(dst + off) =
                                make_uint4(tf32_bits(v[g].x), tf32_bits(v[g].y), tf32_bits(v[g].z), tf32_bits(v[g].w));
                            continue;
                        }
                        uint2 h;
                        h.x = pack_bf16(v[g].x, v[g].y);
                        h.y = pack_bf16(v[g].z, v[g].w);
                        *reinterpret_cast<uint2*>(dst + off) = h;
                        if (SPLIT) {   // residual of the rounding, the lo part
                            const float2 f0 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.x));
                            const float2 f1 = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&h.y));
                            uint2 l;
                            l.x = pack_bf16(v[g].x - f0.x, v[g].y - f0.y);
                            l.y = pack_bf16(v[g].z - f1.x, v[g].w - f1.y);
                            *reinterpret_cast<uint2*>(dst + CPS * NTc * 128 + off) = l;
                        }
                    }
                }
                if (sub == CPS - 1) fence_proxy_async();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&stg_empty[rs.s]);
                    if (sub == CPS - 1) mbar_arrive(&st_full[rb.s]);
                }
                rs.next(a.SS);
                if (sub == CPS - 1) rb.next(a.SB);
            }
            if (!ok) break;
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
            if (!W3(&phi_empty[buf], (use & 1u) ^ 1u, 0x800u)) break;
            cp_async_wait<0>();
            // per cell of the pair tile: 1 - dt sigma_t, dt (sigma_s Phi / sum w + q), neighbour bits
            // (1 left, 2 right, 4 below, 8 above exist; 16 the cell exists), written here and, by
            // st.async completing on the peer's phi_full, into the peer
            const uint32_t pbar = phi_rem + 8u * (uint32_t)buf;
#pragma unroll
            for (int k = 0; k < NOWN; ++k) {
                const int i = col4 + 16 * k;
                if (i >= NR || rsub + RS * i >= NTc) continue;
                float phi = 0.0f;
#pragma unroll
                for (int i2 = 0; i2 < NR; ++i2) phi = i2 == i ? part[i2] : phi;
                const int r = rsub + RS * i;
                const int xx = xbase + (r & (kTW - 1)), yy = ybase + r / kTW;
                float fx = 1.0f, fy = 0.0f;
                int bits = 0;
                if (xx < a.nx && yy < a.ny) {
                    const CellF cl = cst[r];
                    fx = 1.0f - dt * cl.sig_t;
                    fy = dt * (cl.sig_s_over_wsum * phi + cl.q);
                    bits = (xx > 0 ? 1 : 0) | (xx + 1 < a.nx ? 2 : 0) | (yy > 0 ? 4 : 0) | (yy + 1 < a.ny ? 8 : 0) | 16;
                }
                const int c = buf * NT + (int)rank * NTc + r;
                cx[c] = fx;
                cy[c] = fy;
                cb[c] = bits;
                st_async_b32(cx_rem + 4u * (uint32_t)c, __float_as_uint(fx), pbar);
                st_async_b32(cy_rem + 4u * (uint32_t)c, __float_as_uint(fy), pbar);
                st_async_b32(cb_rem + 4u * (uint32_t)c, (uint32_t)bits, pbar);
            }
            __syncwarp();
            if (lane == 0) {
                if (warp == 1) mbar_expect_tx(&phi_full[buf], (uint32_t)NTc * 12u);   // the peer's bytes
                else mbar_arrive(&phi_full[buf]);
            }
        }
    } else {
        // ------------------------------------------------------------------------ epilogue
        const int e = warp - kEpi0;
        const int lq = warp & 3;             // TMEM lane quarter this warp may access
        const int g = e >> 2;                // 0..3
        const int j = MG == 2 ? (g >> 1) : 0;                        // 256-row group
        const int strip = MG == 2 ? (g & 1) : g;
        const int xs = 8 * (strip & 1), ys = MG == 2 ? 0 : 8 * (strip >> 1);
        const int q = 256 * j + 128 * (int)rank + 32 * lq + lane;   // this lane's ordinate
        const bool qlive = q < a.Q;
        const bool warp_pad = 256 * j + 128 * (int)rank + 32 * lq + 31 >= a.Q;   // some lanes are padding
        const float4 o4 = qlive ? __ldg(reinterpret_cast<const float4*>(a.ord) + q) : make_float4(0.f, 0.f, 0.f, 0.f);
        const float ax = fabsf(o4.x), ay = fabsf(o4.y), axy = ax + ay;
        const bool xpos = o4.x > 0.f, ypos = o4.y > 0.f;
        const float dts = a.dts, nge = -dts * o4.w;
        const int nx = a.nx, ny = a.ny;
        const size_t rowstride = (size_t)nx * QP;
        const uint32_t tm_empty0 = mapa_shared(smem_u32(tm_empty), 0);
        const uint32_t phe_loc = mapa_shared(smem_u32(phi_empty), rank);
        const uint32_t phe_rem = mapa_shared(smem_u32(phi_empty), rank ^ 1u);
        const int xedge = xpos ? -1 : 8;      // column of the edge cell (relative to the strip)
        const float2 AX = make_float2(ax, ax), AY = make_float2(ay, ay), NAXY = make_float2(-axy, -axy);
        // upwind weights by side: a_x on the lower or the upper neighbour, zero on the other (a zero
        // weight adds an exact zero, so the sum equals taking the upwind neighbour alone)
        const float cl = xpos ? ax : 0.0f, cr = xpos ? 0.0f : ax, cd = ypos ? ay : 0.0f, cu = ypos ? 0.0f : ay;
        const float2 CL = make_float2(cl, cl), CR = make_float2(cr, cr), CD = make_float2(cd, cd), CU = make_float2(cu, cu);
        const float2 DTS = make_float2(dts, dts), NGE = make_float2(nge, nge);

        for (int T = pair, it = 0; T < total; T += npair, ++it) {
            const int ty = T / a.ntx, tx = T - ty * a.ntx;
            const int x0 = tx * kTW + xs, y0 = ty * TH + ys;   // this warp's strip origin
            const int buf = it & 1;
            const uint32_t use = (uint32_t)(it >> 1);
            const bool interior = !warp_pad && tx * kTW >= 1 && tx * kTW + kTW + 1 <= nx && ty * TH >= 1 &&
                                  ty * TH + TH + 1 <= ny;
            const float* pin = a.in + ((size_t)y0 * nx + x0) * QP + q;   // cell (x0, y0), this ordinate
            float* pout = a.out + ((size_t)y0 * nx + x0) * QP + q;
            const int c0 = buf * NT + ys * kTW + xs;                    // coefficient index of (x0, y0)
            const uint32_t tcol = tmem_base + ((uint32_t)(lq * 32) << 16) +
                                  (uint32_t)(buf * MG * NT + j * NT + ys * kTW + xs);
            if constexpr (HEUN) {
                // Heun stage: the strip in two halves of 4 cells, each walked along its 8 rows.  A row
                // is read with two cells either side (x-stencil), three rows are held ahead of the
                // one updated (y-stencil), zero outside the grid (vacuum) and on padded ordinates.
                // The limited differences take the lane's upwind side:
                //   nu > 0: (psi_i - psi_{i-1}) + (D_i - D_{i-1}) / 2,
                //   nu < 0: (psi_{i+1} - psi_i) - (D_{i+1} - D_i) / 2,   D_i = minmod(psi_i - psi_{i-1}, psi_{i+1} - psi_i),
                // each slope computed once per row and shared by the neighbouring cells.
                const float nux = o4.x, nuy = o4.y, alpha = a.alpha, beta = a.beta;
                const float2 NAX = make_float2(-fabsf(nux), -fabsf(nux)), NAY = make_float2(-fabsf(nuy), -fabsf(nuy));
                const float2 ALPHA = make_float2(alpha, alpha), BETA = make_float2(beta, beta);
                if (alpha != 0.0f && qlive) {
                    // stage 2: psi^n of the strip (the buffer this stage overwrites) has long left L2;
                    // ask for it while the tile's contraction runs (the walk reads it a row ahead)
                    for (int r = 0; r < 8 && y0 + r < ny; ++r)
#pragma unroll
                        for (int i = 0; i < 8; ++i)
                            if (x0 + i < nx)
                                asm volatile("prefetch.global.L2 [%0];" ::"l"(pout + (long)r * (long)rowstride + i * QP));
                }
                int go = 1;
                if (lane == 0) go = W3C(&phi_full[buf], use & 1u, 0x1000u) && W3(&tm_full[buf], use & 1u, 0x2000u);
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) break;
                tc_fence_after();
                // whole stencil (rows y0-2 .. y0+9, cells x0-2 .. x0+9) inside the grid, every lane live:
                // the walk without bounds checks
                const bool inside = !warp_pad && x0 >= 2 && x0 + 10 <= nx && y0 >= 2 && y0 + 10 <= ny;
                auto walk = [&](auto checked_tag) {
                    constexpr bool CK = decltype(checked_tag)::value;
#pragma unroll 1
                for (int hh = 0; hh < 2; ++hh) {
                    const int xh = x0 + 4 * hh;   // first cell of this half
                    // strip row r: its 4 cells (S) or the two cells either side of them (H: xh-2, xh-1,
                    // xh+4, xh+5), zero outside the grid and on padded ordinates; psi^n of its cells
                    // for stage 2 (K), which is the buffer the stage writes: read a row ahead of its
                    // use, by the thread that then overwrites it
                    const float* base = a.in + ((size_t)y0 * nx + xh) * QP + q;   // (xh, y0), this ordinate
                    float* obase = a.out + ((size_t)y0 * nx + xh) * QP + q;
                    auto ld4 = [&](int r, int k0, int k1, int k2, int k3, float (&v)[4]) {
                        const int ks[4] = {k0, k1, k2, k3};
                        const float* p = base + (long)r * (long)rowstride;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if constexpr (CK) {
                                const int yy = y0 + r, xx = xh + ks[i];
                                v[i] = (qlive && yy >= 0 && yy < ny && xx >= 0 && xx < nx) ? __ldg(p + ks[i] * QP) : 0.0f;
                            } else {
                                v[i] = __ldg(p + ks[i] * QP);
                            }
                        }
                    };
                    auto ldS = [&](int r, float (&v)[4]) { ld4(r, 0, 1, 2, 3, v); };
                    auto ldH = [&](int r, float (&v)[4]) { ld4(r, -2, -1, 4, 5, v); };
                    auto ldK = [&](int r, float (&v)[4]) {
                        const float* p = obase + (long)r * (long)rowstride;
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if constexpr (CK) v[i] = (alpha != 0.0f && qlive && y0 + r < ny && xh + i < nx) ? p[i * QP] : 0.0f;
                            else v[i] = alpha != 0.0f ? p[i * QP] : 0.0f;
                        }
                    };
                    float m2S[4], m1S[4], cS[4], cH[4], p1S[4], p1H[4], p2S[4], p2H[4], kc[4];
                    ldS(-2, m2S);
                    ldS(-1, m1S);
                    ldS(0, cS);
                    ldH(0, cH);
                    ldS(1, p1S);
                    ldH(1, p1H);
                    ldS(2, p2S);
                    ldH(2, p2H);
                    ldK(0, kc);
                    // y-slope of the current row, and its difference to the slope of the row below
                    float Dc[4], EyP[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float Dp = minmod3(m1S[i] - m2S[i], cS[i] - m1S[i]);
                        Dc[i] = minmod3(cS[i] - m1S[i], p1S[i] - cS[i]);
                        EyP[i] = Dc[i] - Dp;
                    }
#pragma unroll
                    for (int r = 0; r < 8; ++r) {
                        float p3S[4], p3H[4], kn[4];
                        if (r < 7) {
                            ldS(r + 3, p3S);
                            ldK(r + 1, kn);
                        }
                        if (r < 6) ldH(r + 3, p3H);
                        float y[4];
                        tmem_ld4(tcol + (uint32_t)(r * kTW + 4 * hh), y);
                        // the current row, cells xh-2 .. xh+5
                        const float c[8] = {cH[0], cH[1], cS[0], cS[1], cS[2], cS[3], cH[2], cH[3]};
                        // slopes of the row above (y) and of cells xh-1 .. xh+4 (x), and the differences
                        // of neighbouring slopes: the limited difference on the lane's upwind side is
                        //   (psi - psi_up) + (difference of the slopes on that side) / 2
                        // with the sign of the velocity folded into the coefficient -|nu| (for nu < 0
                        // it is the negated downwind form, so the product is the same number)
                        float Dn[4], EyN[4], Dx[6], Ex[5];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            Dn[i] = minmod3(p1S[i] - cS[i], p2S[i] - p1S[i]);
                            EyN[i] = Dn[i] - Dc[i];
                        }
#pragma unroll
                        for (int k = 1; k <= 6; ++k) Dx[k - 1] = minmod3(c[k] - c[k - 1], c[k + 1] - c[k]);
#pragma unroll
                        for (int j = 0; j < 5; ++j) Ex[j] = Dx[j + 1] - Dx[j];
                        float* po = obase + (long)r * (long)rowstride;
                        const int ci = c0 + r * kTW + 4 * hh;
                        float out[4];
#pragma unroll
                        for (int i = 0; i < 4; i += 2) {
                            float txd[2], tyd[2], st[2];
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const int k = i + u + 2;
                                const float cv = c[k];
                                txd[u] = (cv - (xpos ? c[k - 1] : c[k + 1])) + 0.5f * (xpos ? Ex[k - 2] : Ex[k - 1]);
                                tyd[u] = (cv - (ypos ? m1S[i + u] : p1S[i + u])) + 0.5f * (ypos ? EyP[i + u] : EyN[i + u]);
                                st[u] = operand_value<PR>(cv);
                            }
                            const float2 CV = make_float2(c[i + 2], c[i + 3]);
                            float2 adv = __ffma2_rn(CV, *reinterpret_cast<const float2*>(cx + ci + i),
                                                    *reinterpret_cast<const float2*>(cy + ci + i));
                            adv = __ffma2_rn(NAX, make_float2(txd[0], txd[1]), adv);
                            adv = __ffma2_rn(NAY, make_float2(tyd[0], tyd[1]), adv);
                            adv = __ffma2_rn(DTS, make_float2(y[i], y[i + 1]), adv);
                            adv = __ffma2_rn(NGE, make_float2(st[0], st[1]), adv);
                            const float2 o = __ffma2_rn(ALPHA, make_float2(kc[i], kc[i + 1]), __fmul2_rn(BETA, adv));
                            out[i] = o.x;
                            out[i + 1] = o.y;
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            if constexpr (CK) {
                                if (y0 + r >= ny || xh + i >= nx) continue;
                                if (!qlive) out[i] = 0.0f;
                            }
                            __stcs(po + i * QP, out[i]);
                        }
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            m1S[i] = cS[i];
                            cS[i] = p1S[i];
                            cH[i] = p1H[i];
                            p1S[i] = p2S[i];
                            p1H[i] = p2H[i];
                            if (r < 7) p2S[i] = p3S[i];
                            if (r < 6) p2H[i] = p3H[i];
                            Dc[i] = Dn[i];
                            EyP[i] = EyN[i];
                            if (r < 7) kc[i] = kn[i];
                        }
                    }
                }
                };
                if (inside) walk(std::false_type{});
                else walk(std::true_type{});
            } else if (interior) {
                // rows -1 .. 8 of the strip, row r at rv[r + 1]; edge cell of row r at ev[r + 1]
                float rv[10][8], ev[10];
                auto load_row = [&](int r) {
                    const float* p = pin + (long)r * (long)rowstride;
#pragma unroll
                    for (int i = 0; i < 8; ++i) rv[r + 1][i] = __ldg(p + i * QP);
                    ev[r + 1] = __ldg(p + xedge * QP);
                };
                // halo rows: the one below (Omega_y > 0) or above (Omega_y < 0) the strip
                {
                    const float* p = pin + (ypos ? -(long)rowstride : 8 * (long)rowstride);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float v = __ldg(p + i * QP);
                        rv[0][i] = v;
                        rv[9][i] = v;
                    }
                }
                load_row(0);
                load_row(1);
                load_row(2);
                int go = 1;
                if (lane == 0) go = W3C(&phi_full[buf], use & 1u, 0x1000u) && W3(&tm_full[buf], use & 1u, 0x2000u);
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) break;
                tc_fence_after();
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    if (r + 3 < 8) load_row(r + 3);
                    float y[8];
                    tmem_ld8(tcol + (uint32_t)(r * kTW), y);
                    const float4* cxr = reinterpret_cast<const float4*>(cx + c0 + r * kTW);
                    const float4* cyr = reinterpret_cast<const float4*>(cy + c0 + r * kTW);
                    const float4 xa = cxr[0], xb = cxr[1], ya = cyr[0], yb = cyr[1];
                    const float fxv[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
                    const float fyv[8] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
                    const float* s = rv[r + 1];
                    const float* dn = rv[r];         // row below
                    const float* up = rv[r + 2];     // row above (the halo row for r = 7)
                    float* po = pout + (long)r * (long)rowstride;
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int i0 = 2 * k, i1 = 2 * k + 1;
                        // lower / upper x-neighbours of cells i0, i1 (the row's edge cell stands in at
                        // the ends: it is the side the lane's ordinate looks upwind to, weighted by
                        // cl or cr accordingly)
                        const float xl0 = i0 == 0 ? ev[r + 1] : s[i0 - 1], xr0 = s[i0 + 1];
                        const float xl1 = s[i1 - 1], xr1 = i1 == 7 ? ev[r + 1] : s[i1 + 1];
                        const float2 S = make_float2(s[i0], s[i1]);
                        // the operand of the generator term: psi~ as the contraction saw it (split: psi itself)
                        const float2 ST = PR == kPrBF16
                                              ? __bfloat1622float2(__floats2bfloat162_rn(s[i0], s[i1]))
                                              : make_float2(operand_value<PR>(s[i0]), operand_value<PR>(s[i1]));
                        float2 o = __ffma2_rn(S, __fadd2_rn(make_float2(fxv[i0], fxv[i1]), NAXY),
                                              make_float2(fyv[i0], fyv[i1]));
                        o = __ffma2_rn(CL, make_float2(xl0, xl1), o);
                        o = __ffma2_rn(CR, make_float2(xr0, xr1), o);
                        o = __ffma2_rn(CD, make_float2(dn[i0], dn[i1]), o);
                        o = __ffma2_rn(CU, make_float2(up[i0], up[i1]), o);
                        o = __ffma2_rn(DTS, make_float2(y[i0], y[i1]), o);
                        o = __ffma2_rn(NGE, ST, o);
                        __stcs(po + i0 * QP, o.x);
                        __stcs(po + i1 * QP, o.y);
                    }
                }
            } else {
                // boundary tiles and lanes past Q: every load and store checked against the grid,
                // vacuum (zero) upwind values outside it, zero flux on padded ordinates
                float cur[8], prv[8], nxt[8], edge = 0.0f;
                auto load = [&](int r, float (&v)[8], float& ed) {
                    const int yy = y0 + r;
                    const bool rowok = yy >= 0 && yy < ny;
                    const float* p = pin + (long)r * (long)rowstride;
#pragma unroll
                    for (int i = 0; i < 8; ++i) v[i] = (rowok && x0 + i < nx) ? __ldg(p + i * QP) : 0.0f;
                    const int xe = x0 + xedge;
                    ed = (rowok && xe >= 0 && xe < nx) ? __ldg(p + xedge * QP) : 0.0f;
                };
                float dummy;
                load(-1, prv, dummy);
                load(0, cur, edge);
                float enext = 0.0f;
                int go = 1;
                if (lane == 0) go = W3C(&phi_full[buf], use & 1u, 0x1000u) && W3(&tm_full[buf], use & 1u, 0x2000u);
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) break;
                tc_fence_after();
                for (int r = 0; r < 8; ++r) {
                    load(r + 1, nxt, enext);
                    float y[8];
                    tmem_ld8(tcol + (uint32_t)(r * kTW), y);
                    const int cc = c0 + r * kTW;
                    float* po = pout + (long)r * (long)rowstride;
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const int bits = cb[cc + i];
                        if (!(bits & 16) || q >= QP) continue;
                        if (!qlive) {
                            __stcs(po + i * QP, 0.0f);
                            continue;
                        }
                        float ux = xpos ? (i == 0 ? edge : cur[i - 1]) : (i == 7 ? edge : cur[i + 1]);
                        ux = (bits & (xpos ? 1 : 2)) ? ux : 0.0f;
                        float uy = ypos ? prv[i] : nxt[i];
                        uy = (bits & (ypos ? 4 : 8)) ? uy : 0.0f;
                        const float sf = cur[i];
                        float out = fmaf(sf, cx[cc + i] - axy, cy[cc + i]);
                        out = fmaf(ax, ux, out);
                        out = fmaf(ay, uy, out);
                        out = fmaf(dts, y[i], out);
                        out = fmaf(nge, operand_value<PR>(sf), out);
                        __stcs(po + i * QP, out);
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        prv[i] = cur[i];
                        cur[i] = nxt[i];
                    }
                    edge = enext;
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {   // this warp's accumulator columns and coefficients are read
                mbar_arrive_remote(tm_empty0 + 8u * (uint32_t)buf);
                mbar_arrive_remote(phe_loc + 8u * (uint32_t)buf);
                mbar_arrive_remote(phe_rem + 8u * (uint32_t)buf);
            }
        }
    }

    cp_async_wait<0>();
    __syncthreads();
    cluster_sync();   // neither CTA frees its memory while the pair's MMAs or arrivals may touch it
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, 512);
    }
}

#undef W3
#undef W3C

using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeFn get_encode3() {
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

// Flux [ny][nx][Qp] FP32 as a 3D tensor {Qp, nx, ny}, box {64 ordinates, TW cells, rows}.
bool encode_psi3(CUtensorMap* map, const float* psi, int Qp, int nx, int ny, int rows) {
    EncodeFn enc = get_encode3();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)Qp, (cuuint64_t)nx, (cuuint64_t)ny};
    const cuuint64_t strides[2] = {(cuuint64_t)Qp * 4, (cuuint64_t)Qp * 4 * nx};
    const cuuint32_t box[3] = {64, (cuuint32_t)kTW, (cuuint32_t)rows};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(psi), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// G [Mp][Qp] BF16 as a 5D tensor {64 columns, 128 rows, 2 halves, MG groups, KC chunks}: one box
// {64, 128, 1, MG, CPS} brings one CTA's rows of every 256-row group for CPS 64-column chunks, landing
// as CPS x MG consecutive canonical [128 x 64] K-major tiles (128-byte swizzle), chunk-major.  The
// resident kernel matrix takes single blocks (MG = CPS = 1 in the box).
bool encode_G5(CUtensorMap* map, const __nv_bfloat16* G, int Qp, int MG, int CPS, int box_mg) {
    EncodeFn enc = get_encode3();
    if (!enc) return false;
    const cuuint64_t dims[5] = {64, 128, 2, (cuuint64_t)MG, (cuuint64_t)(Qp / 64)};
    const cuuint64_t strides[4] = {(cuuint64_t)Qp * 2, (cuuint64_t)Qp * 2 * 128, (cuuint64_t)Qp * 2 * 256, 128};
    const cuuint32_t box[5] = {64, 128, 1, (cuuint32_t)box_mg, (cuuint32_t)CPS};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<__nv_bfloat16*>(G), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// G [Mp][Qp] TF32 (FP32 words) as a 5D tensor {32 columns, 128 rows, 2 halves, MG groups, Qp / 32
// chunks}: one box {32, 128, 1, MG, 1} brings one CTA's rows of every 256-row group for one
// 32-column chunk, landing as MG consecutive [128 x 32] K-major tiles of 128-byte rows (128-byte
// swizzle); a 64-ordinate stage takes chunks 2 kc and 2 kc + 1.
bool encode_G5_tf32(CUtensorMap* map, const float* G, int Qp, int MG) {
    EncodeFn enc = get_encode3();
    if (!enc) return false;
    const cuuint64_t dims[5] = {32, 128, 2, (cuuint64_t)MG, (cuuint64_t)(Qp / 32)};
    const cuuint64_t strides[4] = {(cuuint64_t)Qp * 4, (cuuint64_t)Qp * 4 * 128, (cuuint64_t)Qp * 4 * 256, 128};
    const cuuint32_t box[5] = {32, 128, 1, (cuuint32_t)MG, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, const_cast<float*>(G), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int MG, int CPS, int PR>
size_t smem3(int SS, int SB, int nslot) {
    return (size_t)1024 + (size_t)L3<MG, CPS, PR>(SS, SB, SB, nslot).end;
}

// (the split and TF32 layouts are the same size: two parts per chunk, one chunk per stage; BF16X2
// has one operand part)
size_t smem3_for(int MG, int CPS, int pr, int SS, int SB, int nslot) {
    if (pr == kPrX2) return MG == 2 ? smem3<2, 1, kPrX2>(SS, SB, nslot) : smem3<1, 1, kPrX2>(SS, SB, nslot);
    if (pr != kPrBF16) return MG == 2 ? smem3<2, 1, kPrSplit>(SS, SB, nslot) : smem3<1, 1, kPrSplit>(SS, SB, nslot);
    if (MG == 2) return CPS == 2 ? smem3<2, 2, kPrBF16>(SS, SB, nslot) : smem3<2, 1, kPrBF16>(SS, SB, nslot);
    return CPS == 2 ? smem3<1, 2, kPrBF16>(SS, SB, nslot) : smem3<1, 1, kPrBF16>(SS, SB, nslot);
}

// The distinct [128 x 64] blocks of G that the pair's MMAs read, as (even CTA's block, odd CTA's
// block) pairs: a block of group j and chunk kc holds rows 256 j + 128 r .. + 127 (CTA r) and
// columns 64 kc .. 64 kc + 63.  Both CTAs address a pair through one shared-memory slot, so two
// (j, kc) share a slot only when both CTAs' blocks are equal bit for bit.  Fills the 4-bit slot and
// representative tables and returns the number of slots (0 if G could not be read).
int distinct_blocks(const __nv_bfloat16* G, int Qp, int MG, cudaStream_t s, unsigned long long* slots,
                    unsigned long long* reps) {
    const int KC = Qp / 64;
    std::vector<uint16_t> h((size_t)256 * MG * Qp);
    if (cudaMemcpyAsync(h.data(), G, h.size() * 2, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return 0;
    auto same = [&](int a, int b) {   // block indices kc MG + j
        const int ja = a % MG, ka = a / MG, jb = b % MG, kb = b / MG;
        for (int r = 0; r < 256; ++r)
            if (memcmp(&h[(size_t)(256 * ja + r) * Qp + 64 * ka], &h[(size_t)(256 * jb + r) * Qp + 64 * kb], 128))
                return false;
        return true;
    };
    int n = 0;
    *slots = *reps = 0ull;
    for (int idx = 0; idx < KC * MG; ++idx) {
        int sl = -1;
        for (int t = 0; t < n && sl < 0; ++t)
            if (same((int)((*reps >> (4 * t)) & 15u), idx)) sl = t;
        if (sl < 0) {
            sl = n++;
            *reps |= (unsigned long long)idx << (4 * sl);
        }
        *slots |= (unsigned long long)sl << (4 * idx);
    }
    return n;
}

using Tc3Kernel = void (*)(Tc3Args);
template <bool HEUN>
Tc3Kernel kernel3_t(int MG, int CPS, int pr) {
    if (pr == kPrTF32) return MG == 2 ? step_tc3_kernel<2, 1, kPrTF32, HEUN> : step_tc3_kernel<1, 1, kPrTF32, HEUN>;
    if (pr == kPrX2) return MG == 2 ? step_tc3_kernel<2, 1, kPrX2, HEUN> : step_tc3_kernel<1, 1, kPrX2, HEUN>;
    if (pr == kPrSplit) return MG == 2 ? step_tc3_kernel<2, 1, kPrSplit, HEUN> : step_tc3_kernel<1, 1, kPrSplit, HEUN>;
    if (MG == 2) return CPS == 2 ? step_tc3_kernel<2, 2, kPrBF16, HEUN> : step_tc3_kernel<2, 1, kPrBF16, HEUN>;
    return CPS == 2 ? step_tc3_kernel<1, 2, kPrBF16, HEUN> : step_tc3_kernel<1, 1, kPrBF16, HEUN>;
}
Tc3Kernel kernel3(int MG, int CPS, int pr, bool heun) {
    return heun ? kernel3_t<true>(MG, CPS, pr) : kernel3_t<false>(MG, CPS, pr);
}

}  // namespace

struct Tc3Plan {
    int MG = 0, CPS = 2, SS = 0, SB = 0, SA = 0, grid = 0, total = 0, ntx = 0;
    int nslot = 0;                      // resident kernel-matrix blocks (0: the kernel-matrix ring)
    unsigned long long slots = 0, reps = 0;
    int pr = kPrBF16;                   // contraction precision of the instance launched
    size_t smem = 0;
    CUtensorMap tm_psi[2], tm_G, tm_Glo;
    const float* buf[2] = {nullptr, nullptr};
    int nx = 0, ny = 0, Q = 0;
};

bool tc3_supported(int Q, int Qp, int Mp, bool split) {
    (void)Q;
    (void)split;
    return (Qp == 256 || Qp == 512) && Mp == Qp;
}

cudaError_t tc3_plan_create(Tc3Plan** out, const float* buf0, const float* buf1, const TcOperands& ops,
                            int precision, int Q, int Qp, int Mp, int nx, int ny, TcRings want, cudaStream_t stream) {
    *out = nullptr;
    const int pr = precision == ASSN_BF16 ? kPrBF16 : precision == ASSN_BF16X3 ? kPrSplit
                 : precision == ASSN_TF32 ? kPrTF32 : precision == ASSN_BF16X2 ? kPrX2 : -1;
    if (pr < 0 || (pr == kPrTF32 ? !ops.G32 : !ops.G_hi) || ((pr == kPrSplit || pr == kPrX2) && !ops.G_lo))
        return cudaErrorInvalidValue;
    const bool split = pr != kPrBF16;   // two kernel-matrix parts per chunk
    if (!tc3_supported(Q, Qp, Mp, split)) return cudaErrorNotSupported;
    Tc3Plan* p = new Tc3Plan();
    p->MG = Qp / 256;
    p->pr = pr;
    const size_t limit = 227 * 1024;
    // rings as requested (MPR: 64-ordinate chunks per operand / kernel-matrix stage, 1 or 2), else
    // two chunks per stage, two operand and kernel-matrix stages, and as many staging stages as fit,
    // up to four (measured on the 448^2 lattice at 512 ordinates: the staging depth mattered most,
    // two stages 0.30 ms, three or four 0.24 ms; two chunks per stage cut the per-round waits)
    p->CPS = (want.MPR == 1 || split) ? 1 : 2;   // two kernel-matrix parts: one chunk per stage
    p->SS = want.SS ? want.SS : 4;
    p->SB = p->SA = want.SB ? want.SB : (want.SA ? want.SA : 2);
    // the kernel matrix resident (no kernel-matrix ring requested, one BF16 part, not while the
    // stream is being captured: the check reads G back): its distinct blocks, loaded once per
    // launch, when they fit beside two staging stages
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (!want.SA && !split && cudaStreamIsCapturing(stream, &cap) == cudaSuccess &&
        cap == cudaStreamCaptureStatusNone) {
        const int n = distinct_blocks(ops.G_hi, Qp, p->MG, stream, &p->slots, &p->reps);
        if (n > 0 && smem3_for(p->MG, p->CPS, kPrBF16, want.SS ? want.SS : 2, p->SB, n) <= limit) p->nslot = n;
    }
    auto need = [&](int) { return smem3_for(p->MG, p->CPS, p->pr, p->SS, p->SB, p->nslot); };
    if (!want.SS)
        while (p->SS > 2 && need(p->SA) > limit) --p->SS;
    if (need(p->SA) > limit) { delete p; return cudaErrorNotSupported; }
    p->smem = need(p->SA);
    const int TH = (256 / p->MG) / kTW;
    p->nx = nx;
    p->ny = ny;
    p->Q = Q;
    p->ntx = (nx + kTW - 1) / kTW;
    p->total = p->ntx * ((ny + TH - 1) / TH);
    p->buf[0] = buf0;
    p->buf[1] = buf1;
    const bool gmap = pr == kPrTF32 ? encode_G5_tf32(&p->tm_G, ops.G32, Qp, p->MG)
                                    : encode_G5(&p->tm_G, ops.G_hi, Qp, p->MG, p->nslot ? 1 : p->CPS, p->nslot ? 1 : p->MG);
    if (!encode_psi3(&p->tm_psi[0], buf0, Qp, nx, ny, TH / 2) || !encode_psi3(&p->tm_psi[1], buf1, Qp, nx, ny, TH / 2) ||
        !gmap || ((pr == kPrSplit || pr == kPrX2) && !encode_G5(&p->tm_Glo, ops.G_lo, Qp, p->MG, p->CPS, p->MG))) {
        delete p;
        return cudaErrorInvalidValue;
    }
    // one pair per two SMs, as many pairs as the device co-schedules (never more than tiles)
    auto kern = kernel3(p->MG, p->CPS, p->pr, false);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p->smem);
    if (e == cudaSuccess)   // the Heun-stage instance: same layout and shared memory
        e = cudaFuncSetAttribute(kernel3(p->MG, p->CPS, p->pr, true), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)p->smem);
    if (e != cudaSuccess) { delete p; return e; }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int clusters = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * std::max(1, sms / 2), 1, 1);
    cfg.blockDim = dim3(kThreads3, 1, 1);
    cfg.dynamicSmemBytes = p->smem;
    cudaLaunchAttribute attr;
    attr.id = cudaLaunchAttributeClusterDimension;
    attr.val.clusterDim.x = 2;
    attr.val.clusterDim.y = 1;
    attr.val.clusterDim.z = 1;
    cfg.attrs = &attr;
    cfg.numAttrs = 1;
    e = cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg);
    if (e != cudaSuccess || clusters < 1) {
        delete p;
        return e != cudaSuccess ? e : cudaErrorNotSupported;
    }
    p->grid = 2 * std::min(clusters, p->total);
    *out = p;
    return cudaSuccess;
}

void tc3_plan_destroy(Tc3Plan* p) { delete p; }

TcRings tc3_plan_rings(const Tc3Plan* p) {
    TcRings r;
    if (p) {
        r.SS = p->SS;
        r.SB = p->SB;
        r.SA = p->nslot ? 0 : p->SA;   // 0: the kernel matrix is resident
        r.MPR = p->CPS;
    }
    return r;
}

void tc3_plan_describe(const Tc3Plan* p, int* tile_cells, int* stages, int* pairs, size_t* smem) {
    if (tile_cells) *tile_cells = p ? 256 / p->MG : 0;
    if (stages) *stages = p ? p->SA : 0;
    if (pairs) *pairs = p ? p->grid / 2 : 0;
    if (smem) *smem = p ? p->smem : 0;
}

namespace {
cudaError_t launch3(const Tc3Plan* p, int parity, const OrdF* ord, const CellF* cell, const float* w, float dt,
                    float dt_sigma_as, bool heun, const float* keep, float alpha, float beta, unsigned int* err_flag,
                    cudaStream_t s, const float* in_ext = nullptr, float* out_ext = nullptr) {
    if (!p || parity < 0 || parity > 1) return cudaErrorInvalidValue;
    Tc3Args a;
    memset(&a, 0, sizeof a);
    a.tm_psi = p->tm_psi[parity];
    a.tm_G = p->tm_G;
    a.tm_Glo = p->pr == kPrSplit || p->pr == kPrX2 ? p->tm_Glo : p->tm_G;
    a.in = p->buf[parity];
    a.out = const_cast<float*>(p->buf[parity ^ 1]);
    a.ord = ord;
    a.cell = cell;
    a.w = w;
    a.err = err_flag;
    a.nx = p->nx;
    a.ny = p->ny;
    a.Q = p->Q;
    a.ntx = p->ntx;
    a.total = p->total;
    a.SS = p->SS;
    a.SB = p->SB;
    a.SA = p->SA;
    a.nslot = p->nslot;
    a.slots = p->slots;
    a.reps = p->reps;
    a.dt = dt;
    a.dts = dt_sigma_as;
    a.keep = keep;
    a.alpha = alpha;
    a.beta = beta;
    if (in_ext) {   // caller-owned buffers of the same layout: a tensor map of this input
        if (!encode_psi3(&a.tm_psi, in_ext, 256 * p->MG, p->nx, p->ny, (256 / p->MG) / kTW / 2))
            return cudaErrorInvalidValue;
        a.in = in_ext;
        a.out = out_ext;
    }
    kernel3(p->MG, p->CPS, p->pr, heun)<<<p->grid, kThreads3, p->smem, s>>>(a);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_step_tc3(const Tc3Plan* p, int parity, const OrdF* ord, const CellF* cell, const float* w,
                            float dt, float dt_sigma_as, unsigned int* err_flag, cudaStream_t s) {
    return launch3(p, parity, ord, cell, w, dt, dt_sigma_as, false, nullptr, 0.0f, 1.0f, err_flag, s);
}

cudaError_t launch_heun_stage_tc3(const Tc3Plan* p, int parity, const OrdF* ord, const CellF* cell, const float* w,
                                  float dt, float dt_sigma_as, const float* keep, float alpha, float beta,
                                  unsigned int* err_flag, cudaStream_t s) {
    return launch3(p, parity, ord, cell, w, dt, dt_sigma_as, true, keep, alpha, beta, err_flag, s);
}

cudaError_t launch_step_tc3_buffers(const Tc3Plan* p, const float* in, float* out, const OrdF* ord,
                                    const CellF* cell, const float* w, float dt, float dt_sigma_as,
                                    unsigned int* err_flag, cudaStream_t s) {
    if (!in || !out || ((uintptr_t)in & 15u) || ((uintptr_t)out & 3u)) return cudaErrorInvalidValue;
    return launch3(p, 0, ord, cell, w, dt, dt_sigma_as, false, nullptr, 0.0f, 1.0f, err_flag, s, in, out);
}

}  // namespace assn
