// Tensor-core (tcgen05) Legendre synthesis and analysis with BF16 hi + lo
// split operands and FP32 accumulation in tensor memory.
//
// Per order m and parity of K - m both Legendre steps of the RHS (Sec. 4.2:
// the evaluation of Eq. (app_soln_rep) on the Gauss latitudes, and the
// projection of Eq. (disc_vec_orth_proj) after the longitude transform) are
// dense contractions with the table block Pt_K^m(x_p):
//     synthesis  g[p][c] = sum_K Pt_K^m(x_p) b[K][c]
//     analysis   H[K][c] = sum_p Pt_K^m(x_p) S[p][c]   (S = hemispheric sum / difference)
// A = table tile (128 rows x 64 of the contracted index, K-major, 128-byte
// swizzle, by TMA from one tensor map per (m, parity) block; rows past the
// block come back zero-filled and are not read from HBM).  B = 16 x 64 tile
// whose rows hold the hi parts (rows 0 .. 2F-1) and lo parts (rows 2F ..
// 4F-1) of the F real columns.  Two MMAs per K step into two accumulators,
//     D1 = A_hi B,   D2 = A_lo B,
// give  result = D1[hi] + D1[lo] + D2[hi] + D2[lo]
//              = A_hi B_hi + A_hi B_lo + A_lo B_hi + A_lo B_lo,
// the product of the FP32-accurate split operands, accumulated in FP32.
//
// Synthesis: the B tiles are written ahead by k_prep_tc (one 2 KB tile per
// (m, parity, K tile)) and arrive with every A stage by bulk copy; warp 0 is
// the TMA producer, warp 1 issues the MMAs, warps 2-5 drain the accumulators.
// Analysis: warps 2-5 build B from the weighted Fourier profiles in 16-byte
// swizzle chunks, warps 6-9 drain the accumulators, so that neither stalls the
// MMA issue behind the other.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "f64cvt.h"
#include "finish.cuh"
#include "internal.h"
#include "tc.cuh"

namespace sph {

constexpr int TC_TILE_M = 128;    // rows per MMA tile
constexpr int TC_TILE_K = 64;     // K per smem tile (128 bytes of bf16)
constexpr int TC_N = 16;          // accumulator columns (B rows)
constexpr int TC_ATILE = TC_TILE_M * TC_TILE_K * 2;   // 16 KB

// 8 bf16 (hi or lo parts of v[0..7]) packed for one 16-byte swizzle chunk
__device__ __forceinline__ uint4 pack_hi(const float* v) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        w[i] = *reinterpret_cast<const uint32_t*>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ uint4 pack_lo(const float* v) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float a = v[2 * i], b = v[2 * i + 1];
        const float la = a - __bfloat162float(__float2bfloat16_rn(a));
        const float lb = b - __bfloat162float(__float2bfloat16_rn(b));
        const __nv_bfloat162 l = __floats2bfloat162_rn(la, lb);
        w[i] = *reinterpret_cast<const uint32_t*>(&l);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}
// byte offset of the 16-byte chunk q (K = 8q .. 8q+7) of row r in a swizzled tile
__device__ __forceinline__ uint32_t sw128_chunk(int r, int q) {
    return uint32_t(r) * 128u + (uint32_t(q ^ (r & 7)) << 4);
}

// Analysis items: tiles of 128 consecutive table rows (the (m, parity) blocks
// packed back to back in degree order), each with up to 32 / (4 NF) pieces =
// the blocks it overlaps.  Piece j owns B columns 4 NF j .. 4 NF j + 4 NF - 1
// (hi parts, then lo parts) and the tile rows [s, e); the MMA computes all
// columns for all rows and the epilogue keeps the columns of each row's piece.
struct TcAnaArgs {
    const CUtensorMap* map_hi;   // whole table [n_ext][nh], box 64 x 128 (FIN: 8 maps, boxes 64 x 16 (j + 1))
    const CUtensorMap* map_lo;
    const int4* items;           // (first table row, first piece, piece count, N | first K tile << 16 | FIN box j << 24)
    const int* item_off;         // per CTA
    const int4* pieces;          // (m, parity, s, e): rows [s, e) of the item's tile
    const float* gana;           // [NF][N+1][nlat] complex float (m-major)
    float* hana;                 // [n_ext][2 NF]
    unsigned* status;
    int N, nh, nlat, nkt, n_ext;
    // FIN (the RHS recombination and update in the epilogue): per item, its
    // order group (first table row, first order, end order, last item of the
    // group), and the finish's operands
    const int4* og;
    const double2* alpha;
    const double2* forcing;
    double2* out;
    const float4* finc;
    double nu, omega_d;
    int srows;                   // rows of one stage buffer (max(2 (N + 2), 128))
    // FIN, direct-output calls: CTAs done, and the mapped host flag the last one sets to done_ticket
    unsigned* done_cnt;
    unsigned long long* done_flag;
    unsigned long long done_ticket;
};

constexpr int TC_ANA_NS = 5;                   // A stages
constexpr int TC_ANA_NS_FIN = 4;               // A stages of the RHS form (its shared memory holds two stage buffers)

// Table tiles whose entries are all below TC_SKIP in magnitude are not read:
// near the poles Pt_K^m decays like sin(theta)^m below its turning point
// sin(theta) = m / (K + 1/2), so at high order whole tiles of the polar
// latitudes are negligible (about a tenth of the table at L = 511).  A
// skipped term changes an output by at most TC_SKIP times the sum of the
// skipped coefficients' magnitudes, six orders below the BF16 split's own
// rounding (~1e-5).
constexpr double TC_SKIP = 1e-11;
constexpr int TC_ANA_BROWS = 32;               // B rows (N) per item at most
constexpr int TC_ANA_BTILE = TC_ANA_BROWS * TC_TILE_K * 2;   // 4 KB per K tile
constexpr int TC_ANA_COLS = 128;               // TMEM: 2 buffers x 64 columns

// FIN: items are order-aligned tiles grouped by order (each CTA takes whole
// groups); the epilogue keeps a group's projection rows in shared memory and
// after the group's last tile computes the packed entries of F for its
// orders (the recombination and diagonal update, Sec. 3), so the RHS needs
// no separate finish kernel.
template <int NF, bool FIN = false>
__global__ void __launch_bounds__(FIN ? 448 : 320, 1) k_ana_tc(TcAnaArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~uintptr_t(1023));
    constexpr int RP = 4 * NF;                                    // B rows per piece
    constexpr int ANS = FIN ? TC_ANA_NS_FIN : TC_ANA_NS;          // A stages
    unsigned char* A_hi = smem;                                   // NS x 16 KB
    unsigned char* A_lo = A_hi + ANS * TC_ATILE;            // NS x 16 KB
    unsigned char* Bt = A_lo + ANS * TC_ATILE;              // 2 bufs x nkt x 4 KB
    uint64_t* bars = reinterpret_cast<uint64_t*>(Bt + 2 * a.nkt * TC_ANA_BTILE);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + ANS;
    uint64_t* b_full = bars + 2 * ANS;
    uint64_t* b_empty = b_full + 2;
    uint64_t* acc_full = b_full + 4;
    uint64_t* acc_empty = b_full + 6;
    uint64_t* st_full = b_full + 8;                               // FIN: an order group's rows staged
    uint64_t* st_empty = st_full + 2;                             // FIN: its F written, buffer free
    uint64_t* st_half = st_empty + 2;                             // FIN: the group's first order staged
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(FIN ? st_half + 2 : b_full + 8);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    float* stage = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(bars) + 256);   // FIN: 2 x [srows][4]

    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int N = a.N, nh = a.nh, nlat = a.nlat, nkt = a.nkt;
    // B rows past the pieces of an item are never read back; start them at zero
    for (int i = threadIdx.x; i < 2 * nkt * TC_ANA_BTILE / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(Bt)[i] = make_uint4(0u, 0u, 0u, 0u);
    fence_proxy_async_smem();
    if (threadIdx.x == 0) {
        for (int s = 0; s < ANS; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&b_full[b], 128);
            mbar_init(&b_empty[b], 1);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
            if constexpr (FIN) {
                mbar_init(&st_full[b], 128);
                mbar_init(&st_empty[b], 128);
                mbar_init(&st_half[b], 128);
            }
        }
        *abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TC_ANA_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_launch();
    const uint32_t tmem = *tmem_slot;
    const int ib = a.item_off[blockIdx.x], nI = a.item_off[blockIdx.x + 1] - ib;

    if (warp == 0) {
        if (lane == 0) {
            // the tables do not depend on the predecessor: stream them right away
            const uint64_t pol = policy_evict_first();
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int4 itm = a.items[ib + i];
                // FIN: the box height of the item's rows (16 (bj + 1)) and its map
                const int bj = FIN ? (itm.w >> 24) & 7 : 0;
                const uint32_t abytes = uint32_t(2 * TC_TILE_K * 2 * (FIN ? 16 * (bj + 1) : TC_TILE_M));
                for (int kt = (itm.w >> 16) & 0xFF; kt < nkt; ++kt, ++it) {
                    const int s = it % ANS;
                    if (it >= ANS && !mbar_wait(&a_empty[s], ((it / ANS) - 1) & 1, abort, a.status))
                        continue;
                    if (*abort) continue;
                    mbar_arrive_expect_tx(&a_full[s], abytes);
                    tma_load_2d(A_hi + s * TC_ATILE, a.map_hi + bj, kt * TC_TILE_K, itm.x, &a_full[s], pol);
                    tma_load_2d(A_lo + s * TC_ATILE, a.map_lo + bj, kt * TC_TILE_K, itm.x, &a_full[s], pol);
                }
            }
            for (int k = it - ANS; k < it; ++k)
                if (k >= 0) mbar_wait(&a_full[k % ANS], (k / ANS) & 1, abort, a.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int4 itm = a.items[ib + i];
                const uint32_t idesc = idesc_bf16(TC_TILE_M, itm.w & 0xFFFF);
                const int kt0 = (itm.w >> 16) & 0xFF;
                const int buf = i & 1, use = i >> 1;
                bool ok = mbar_wait(&b_full[buf], use & 1, abort, a.status);
                if (i >= 2) ok = mbar_wait(&acc_empty[buf], (use - 1) & 1, abort, a.status) && ok;
                tc_fence_after();
                const uint32_t d = tmem + uint32_t(buf * 64);
                for (int kt = kt0; kt < nkt; ++kt, ++it) {
                    const int s = it % ANS;
                    const bool okA = mbar_wait(&a_full[s], (it / ANS) & 1, abort, a.status);
                    tc_fence_after();
                    if (ok && okA && !*abort) {
                        const unsigned char* bt = Bt + (buf * nkt + kt) * TC_ANA_BTILE;
#pragma unroll
                        for (int kk = 0; kk < TC_TILE_K / 16; ++kk) {
                            const uint64_t bd = sdesc_sw128(bt + kk * 32);
                            mma_bf16(d, sdesc_sw128(A_hi + s * TC_ATILE + kk * 32), bd, idesc, (kt > kt0) || kk != 0);
                            mma_bf16(d, sdesc_sw128(A_lo + s * TC_ATILE + kk * 32), bd, idesc, 1);
                        }
                    }
                    mma_commit(&a_empty[s]);
                }
                mma_commit(&acc_full[buf]);
                mma_commit(&b_empty[buf]);
            }
            if (nI > 0) mbar_wait(&acc_full[(nI - 1) & 1], ((nI - 1) >> 1) & 1, abort, a.status);
        }
    } else if (warp < 6) {
        // B builders: task (piece, K tile, chunk q of 8 latitudes, field f)
        pdl_wait();
        const int ht = threadIdx.x - 64;
        const size_t ld = size_t(N + 1);
        for (int i = 0; i < nI; ++i) {
            const int buf = i & 1;
            if (i >= 2) mbar_wait(&b_empty[buf], ((i >> 1) - 1) & 1, abort, a.status);
            const int4 itm = a.items[ib + i];
            const int kt0 = (itm.w >> 16) & 0xFF;
            const int per_piece = (nkt - kt0) * 8 * NF;
            for (int task = ht; task < itm.z * per_piece; task += 128) {
                const int j = task / per_piece, tl = task % per_piece;
                const int4 pc = a.pieces[itm.y + j];
                const int m = pc.x, par = pc.y;
                const int f = tl % NF, q = (tl / NF) & 7, kt = kt0 + tl / (8 * NF);
                const int p0 = kt * TC_TILE_K + q * 8;
                const float* g = a.gana + (size_t(f) * ld + m) * size_t(nlat) * 2;
                float nv[16], sv[16];
                if (p0 + 8 <= nh) {
                    const float4* gn = reinterpret_cast<const float4*>(g + size_t(p0) * 2);
                    const float4* gs = reinterpret_cast<const float4*>(g + size_t(nlat - 8 - p0) * 2);
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const float4 x = gn[u], y = gs[u];
                        nv[4 * u] = x.x; nv[4 * u + 1] = x.y; nv[4 * u + 2] = x.z; nv[4 * u + 3] = x.w;
                        sv[4 * u] = y.x; sv[4 * u + 1] = y.y; sv[4 * u + 2] = y.z; sv[4 * u + 3] = y.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int p = p0 + e, pr = nlat - 8 - p0 + e;
                        const bool in = p < nh;
                        nv[2 * e] = in ? g[2 * size_t(p)] : 0.f;
                        nv[2 * e + 1] = in ? g[2 * size_t(p) + 1] : 0.f;
                        const bool ins = (nlat - 1 - pr) < nh && pr >= 0;
                        sv[2 * e] = ins ? g[2 * size_t(pr)] : 0.f;
                        sv[2 * e + 1] = ins ? g[2 * size_t(pr) + 1] : 0.f;
                    }
                }
                // latitude p0 + e pairs with its mirror nlat - 1 - p0 - e = sv entry 7 - e
                float re[8], im[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const float sr = sv[2 * (7 - e)], si = sv[2 * (7 - e) + 1];
                    re[e] = par ? nv[2 * e] - sr : nv[2 * e] + sr;
                    im[e] = par ? nv[2 * e + 1] - si : nv[2 * e + 1] + si;
                }
                unsigned char* tile = Bt + (buf * nkt + kt) * TC_ANA_BTILE;
                const int r0 = RP * j;
                *reinterpret_cast<uint4*>(tile + sw128_chunk(r0 + 2 * f, q)) = pack_hi(re);
                *reinterpret_cast<uint4*>(tile + sw128_chunk(r0 + 2 * f + 1, q)) = pack_hi(im);
                *reinterpret_cast<uint4*>(tile + sw128_chunk(r0 + 2 * NF + 2 * f, q)) = pack_lo(re);
                *reinterpret_cast<uint4*>(tile + sw128_chunk(r0 + 2 * NF + 2 * f + 1, q)) = pack_lo(im);
            }
            fence_proxy_async_smem();
            mbar_arrive(&b_full[buf]);
        }
    } else if (warp < 10) {
        // epilogue: TMEM lanes of this warp's quarter -> projection rows
        // (FIN: into the stage buffer of the CTA's g-th order group, g & 1)
        pdl_wait();
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;               // tile row of this lane
        int g = 0;
        bool new_group = true;
        for (int i = 0; i < nI; ++i) {
            const int4 itm = a.items[ib + i];
            const int buf = i & 1;
            if (FIN && new_group && g >= 2) mbar_wait(&st_empty[g & 1], ((g >> 1) - 1) & 1, abort, a.status);
            new_group = false;
            float* sg = stage + (g & 1) * a.srows * 2 * NF;
            const bool ok = mbar_wait(&acc_full[buf], (i >> 1) & 1, abort, a.status);
            tc_fence_after();
            const int row = itm.x + r;
            for (int j = 0; j < itm.z; ++j) {
                const int4 pc = a.pieces[itm.y + j];
                if (pc.w <= quarter * 32 || pc.z >= quarter * 32 + 32) continue;   // warp-uniform
                float v[16];
                tmem_ld16(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(buf * 64 + RP * j), v);
                if (ok && r >= pc.z && r < pc.w && row < a.n_ext && !*abort) {
                    if constexpr (FIN) {
                        const int sr = row - a.og[ib + i].x;
#pragma unroll
                        for (int c = 0; c < 2 * NF; ++c) sg[sr * 2 * NF + c] = v[c] + v[2 * NF + c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 2 * NF; ++c)
                            a.hana[size_t(row) * 2 * NF + c] = v[c] + v[2 * NF + c];
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);
            if constexpr (FIN) {
                // a group of two orders releases its first order's finish
                // once that order's last row is staged (other groups with
                // their last tile): the finish of a CTA's last group is
                // its tail after the last MMA
                const int4 og = a.og[ib + i];
                const int end0 = ext_off(N, og.y + 1) - 1;
                const bool first = og.z - og.y == 2
                                       ? itm.x <= end0 && end0 < itm.x + 16 * (((itm.w >> 24) & 7) + 1)
                                       : og.w != 0;
                if (first) mbar_arrive(&st_half[g & 1]);
                if (og.w) {
                    mbar_arrive(&st_full[g & 1]);   // the group's rows are staged
                    ++g;
                    new_group = true;
                }
            }
        }
    } else if constexpr (FIN) {
        // finish warps (10 .. 13): F for the orders of each staged group, one
        // packed entry per thread at a time (the recombination and diagonal
        // update of finish32_entry), while the epilogue stages the next group
        pdl_wait();   // alpha and the forcing may be the predecessor's output
        const int ft = int(threadIdx.x) - 320;
        int g = 0;
        for (int i = 0; i < nI; ++i) {
            const int4 og = a.og[ib + i];
            if (!og.w) continue;
            mbar_wait(&st_half[g & 1], (g >> 1) & 1, abort, a.status);
            const float* sg = stage + (g & 1) * a.srows * 2 * NF;
            const bool two = og.z - og.y == 2;
            if (!two) mbar_wait(&st_full[g & 1], (g >> 1) & 1, abort, a.status);
            if (!*abort) {
                for (int m = og.y; m < og.z; ++m) {
                    // the second order of a two-order group: all rows staged
                    if (two && m > og.y) mbar_wait(&st_full[g & 1], (g >> 1) & 1, abort, a.status);
                    if (*abort) break;
                    const int lo = m > 0 ? m : 1, pk = packed_off(N, m) - lo;
                    // four entries per thread at a time, their operands loaded
                    // first: one load latency per four entries (the group's
                    // finish is the CTA's tail after its last MMA)
                    for (int L0 = lo + ft; L0 <= N; L0 += 4 * 128) {
                        double2 al[4], fo[4];
                        float4 fc[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int L = L0 + 128 * u, pi = pk + L;
                            if (L <= N) {
                                al[u] = a.alpha[pi];
                                fc[u] = a.finc[pi];
                                fo[u] = a.forcing ? a.forcing[pi] : make_double2(0.0, 0.0);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const int L = L0 + 128 * u, pi = pk + L;
                            if (L > N) break;
                            const float* hL = sg + (ext_row(N, m, L) - og.x) * 2 * NF;
                            const float* hU = sg + (ext_row(N, m, L + 1) - og.x) * 2 * NF;
                            const float* hD = L - 1 >= m ? sg + (ext_row(N, m, L - 1) - og.x) * 2 * NF : nullptr;
                            a.out[pi] = finish32_entry(0, L, m, fc[u], hL, hU, hD, al[u], fo[u], a.nu, a.omega_d);
                        }
                    }
                }
            }
            mbar_arrive(&st_empty[g & 1]);
            ++g;
        }
    }
    // direct-output calls: every thread's writes of F reach the system
    // before the CTA counts itself done
    if (FIN && a.done_flag) __threadfence_system();
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TC_ANA_COLS);
    }
    if constexpr (FIN) {
        // the last CTA to finish reports the call complete in mapped host memory
        if (a.done_flag && threadIdx.x == 0 && atomicAdd(a.done_cnt, 1u) == gridDim.x - 1) {
            *a.done_cnt = 0u;
            __threadfence_system();
            *reinterpret_cast<volatile unsigned long long*>(a.done_flag) = a.done_ticket;
        }
    }
}

// ---------------------------------------------------------------------------
// batched analysis (instances of one truncation)
//
// k_ana_prep writes, per instance, block (m, parity) and K tile of 64
// latitudes, the B rows of the analysis as one 1 KB swizzled tile: rows
// 2f, 2f+1 = hi parts of Re, Im of S_f(p) = G_f(p) +- G_f(p') (the
// hemispheric sum for even, difference for odd K - m), rows 4+2f, 5+2f = lo
// parts.  Eight rows make one 128-byte swizzle atom, so the tile is valid at
// any 8-row offset of a B operand.
// k_ana_tc_b streams each 128-row tile of consecutive table rows once per
// item = (tile, <= 32 slots of (overlapped block, instance)); each stage
// brings A_hi, A_lo by TMA and the slots' S tiles by bulk copy into rows
// 8 slot .. 8 slot + 7 of B, so one MMA (N = 8 slots) serves every slot.

// Thread = (instance, order m, K tile, chunk q of 8 latitudes, field f): it
// reads the 8 northern latitudes and their mirrors with 16-byte loads and
// writes both parities' tiles, S = G(p) + G(p') to block 2m and G(p) - G(p')
// to block 2m + 1; consecutive threads take consecutive latitude chunks.
__global__ void __launch_bounds__(128) k_ana_prep(const float* __restrict__ gana, size_t sa, unsigned char* __restrict__ stiles,
                                                  int N, int nh, int nlat, int nkt) {
    pdl_launch();
    pdl_wait();
    const int inst = blockIdx.y;
    const int nblk = 2 * (N + 1);
    const int t = blockIdx.x * 128 + threadIdx.x;   // (m, kt, f, q)
    if (t >= (N + 1) * nkt * 16) return;
    const int q = t & 7, f = (t >> 3) & 1, kt = (t >> 4) % nkt, m = (t >> 4) / nkt;
    const float* g = gana + size_t(inst) * sa + (size_t(f) * (N + 1) + m) * size_t(nlat) * 2;
    const int p0 = kt * TC_TILE_K + q * 8;
    float nv[16], sv[16];
    if (p0 + 8 <= nh) {
        const float4* gn = reinterpret_cast<const float4*>(g + size_t(p0) * 2);
        const float4* gs = reinterpret_cast<const float4*>(g + size_t(nlat - 8 - p0) * 2);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 x = __ldcs(gn + u), y = __ldcs(gs + u);
            nv[4 * u] = x.x; nv[4 * u + 1] = x.y; nv[4 * u + 2] = x.z; nv[4 * u + 3] = x.w;
            sv[4 * u] = y.x; sv[4 * u + 1] = y.y; sv[4 * u + 2] = y.z; sv[4 * u + 3] = y.w;
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int p = p0 + e, pr = nlat - 8 - p0 + e;
            const bool in = p < nh;
            nv[2 * e] = in ? g[2 * size_t(p)] : 0.f;
            nv[2 * e + 1] = in ? g[2 * size_t(p) + 1] : 0.f;
            const bool ins = (nlat - 1 - pr) < nh && pr >= 0;
            sv[2 * e] = ins ? g[2 * size_t(pr)] : 0.f;
            sv[2 * e + 1] = ins ? g[2 * size_t(pr) + 1] : 0.f;
        }
    }
    // latitude p0 + e pairs with its mirror nlat - 1 - p0 - e = sv entry 7 - e
    float er[8], ei[8], odr[8], odi[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float sr = sv[2 * (7 - e)], si = sv[2 * (7 - e) + 1];
        er[e] = nv[2 * e] + sr;
        ei[e] = nv[2 * e + 1] + si;
        odr[e] = nv[2 * e] - sr;
        odi[e] = nv[2 * e + 1] - si;
    }
    unsigned char* te = stiles + ((size_t(inst) * nblk + 2 * m) * nkt + kt) * 1024;
    unsigned char* to = te + size_t(nkt) * 1024;
    *reinterpret_cast<uint4*>(te + sw128_chunk(2 * f, q)) = pack_hi(er);
    *reinterpret_cast<uint4*>(te + sw128_chunk(2 * f + 1, q)) = pack_hi(ei);
    *reinterpret_cast<uint4*>(te + sw128_chunk(4 + 2 * f, q)) = pack_lo(er);
    *reinterpret_cast<uint4*>(te + sw128_chunk(5 + 2 * f, q)) = pack_lo(ei);
    *reinterpret_cast<uint4*>(to + sw128_chunk(2 * f, q)) = pack_hi(odr);
    *reinterpret_cast<uint4*>(to + sw128_chunk(2 * f + 1, q)) = pack_hi(odi);
    *reinterpret_cast<uint4*>(to + sw128_chunk(4 + 2 * f, q)) = pack_lo(odr);
    *reinterpret_cast<uint4*>(to + sw128_chunk(5 + 2 * f, q)) = pack_lo(odi);
}

struct TcAnaBArgs {
    const CUtensorMap* map_hi;   // whole table [n_ext][nh], box 64 x 128
    const CUtensorMap* map_lo;
    const int4* items;           // (tile, first slot, slot count, N)
    const int* item_off;
    const int4* slots;           // (m, parity, instance, rows s | e << 16 within the tile)
    const unsigned char* stiles; // [instance][block][kt] 1 KB
    float* hana;                 // instance i: hana + i * sh floats, [n_ext][4]
    size_t sh;
    unsigned* status;
    int N, nkt, n_ext;
};

constexpr int TC_ANAB_NS = 3;                  // stages of A (32 KB) + B (<= 32 KB)
constexpr int TC_ANAB_BBYTES = 256 * 128;      // B: up to 256 rows

__global__ void __launch_bounds__(192, 1) k_ana_tc_b(TcAnaBArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~uintptr_t(1023));
    unsigned char* A_hi = smem;
    unsigned char* A_lo = A_hi + TC_ANAB_NS * TC_ATILE;
    unsigned char* Bs = A_lo + TC_ANAB_NS * TC_ATILE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + TC_ANAB_NS * TC_ANAB_BBYTES);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + TC_ANAB_NS;
    uint64_t* acc_full = bars + 2 * TC_ANAB_NS;
    uint64_t* acc_empty = acc_full + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 4);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    const int nkt = a.nkt, nblk = 2 * (a.N + 1);
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_ANAB_NS; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        *abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 512);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    pdl_launch();
    const uint32_t tmem = *tmem_slot;
    const int ib = a.item_off[blockIdx.x], nI = a.item_off[blockIdx.x + 1] - ib;

    if (warp == 0) {
        // lane 0 waits for the slot and posts the byte count; every lane then
        // issues the bulk copy of one slot's S tile (lane 0 also the A tiles)
        pdl_wait();
        // the table tile is read again by the tile's other instance items (an
        // ensemble bucket's table is a few MB): keep it in L2; the S tiles are
        // read once
        const uint64_t pol = policy_evict_last();
        const uint64_t polb = policy_evict_first();
        int it = 0;
        for (int i = 0; i < nI; ++i) {
            const int4 itm = a.items[ib + i];
            int4 sl = make_int4(0, 0, 0, 0);
            if (lane < itm.z) sl = a.slots[itm.y + lane];
            for (int kt = itm.w >> 16; kt < nkt; ++kt, ++it) {
                const int s = it % TC_ANAB_NS;
                int go = 0;
                if (lane == 0) {
                    const bool ok = it < TC_ANAB_NS || mbar_wait(&a_empty[s], ((it / TC_ANAB_NS) - 1) & 1, abort, a.status);
                    go = ok && !*abort;
                    if (go) mbar_arrive_expect_tx(&a_full[s], uint32_t(2 * TC_ATILE + itm.z * 1024));
                }
                go = __shfl_sync(0xffffffffu, go, 0);
                if (!go) continue;
                if (lane == 0) {
                    tma_load_2d(A_hi + s * TC_ATILE, a.map_hi, kt * TC_TILE_K, itm.x * TC_TILE_M, &a_full[s], pol);
                    tma_load_2d(A_lo + s * TC_ATILE, a.map_lo, kt * TC_TILE_K, itm.x * TC_TILE_M, &a_full[s], pol);
                }
                if (lane < itm.z) {
                    const unsigned char* src = a.stiles + ((size_t(sl.z) * nblk + 2 * sl.x + sl.y) * nkt + kt) * 1024;
                    bulk_g2s(Bs + s * TC_ANAB_BBYTES + lane * 1024, src, 1024, &a_full[s], polb);
                }
            }
        }
        if (lane == 0)
            for (int k = it - TC_ANAB_NS; k < it; ++k)
                if (k >= 0) mbar_wait(&a_full[k % TC_ANAB_NS], (k / TC_ANAB_NS) & 1, abort, a.status);
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int4 itm = a.items[ib + i];
                const uint32_t idesc = idesc_bf16(TC_TILE_M, itm.w & 0xFFFF);
                const int kt0 = itm.w >> 16;
                const int buf = i & 1, use = i >> 1;
                bool ok = true;
                if (i >= 2) ok = mbar_wait(&acc_empty[buf], (use - 1) & 1, abort, a.status);
                tc_fence_after();
                const uint32_t d = tmem + uint32_t(buf * 256);
                for (int kt = kt0; kt < nkt; ++kt, ++it) {
                    const int s = it % TC_ANAB_NS;
                    const bool okA = mbar_wait(&a_full[s], (it / TC_ANAB_NS) & 1, abort, a.status);
                    tc_fence_after();
                    if (ok && okA && !*abort) {
#pragma unroll
                        for (int kk = 0; kk < TC_TILE_K / 16; ++kk) {
                            const uint64_t bd = sdesc_sw128(Bs + s * TC_ANAB_BBYTES + kk * 32);
                            mma_bf16(d, sdesc_sw128(A_hi + s * TC_ATILE + kk * 32), bd, idesc, (kt > kt0) || kk != 0);
                            mma_bf16(d, sdesc_sw128(A_lo + s * TC_ATILE + kk * 32), bd, idesc, 1);
                        }
                    }
                    mma_commit(&a_empty[s]);
                }
                mma_commit(&acc_full[buf]);
            }
            if (nI > 0) mbar_wait(&acc_full[(nI - 1) & 1], ((nI - 1) >> 1) & 1, abort, a.status);
        }
    } else {
        // epilogue: slot j of the item -> columns 8 j .. 8 j + 7 (hi, then lo parts)
        pdl_wait();
        const int quarter = warp & 3;
        const int r = quarter * 32 + lane;
        for (int i = 0; i < nI; ++i) {
            const int4 itm = a.items[ib + i];
            const int buf = i & 1;
            const bool ok = mbar_wait(&acc_full[buf], (i >> 1) & 1, abort, a.status);
            tc_fence_after();
            const int row = itm.x * TC_TILE_M + r;
            for (int j = 0; j < itm.z; ++j) {
                const int4 sl = a.slots[itm.y + j];
                const int rs = sl.w & 0xFFFF, re = sl.w >> 16;
                if (re <= quarter * 32 || rs >= quarter * 32 + 32) continue;   // warp-uniform
                float v[8];
                tmem_ld8(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(buf * 256 + 8 * j), v);
                if (ok && r >= rs && r < re && row < a.n_ext && !*abort) {
                    float4 h = make_float4(v[0] + v[4], v[1] + v[5], v[2] + v[6], v[3] + v[7]);
                    *reinterpret_cast<float4*>(a.hana + size_t(sl.z) * a.sh + size_t(row) * 4) = h;
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// coefficient sets of the synthesis
//
// zeta: lam^{1/2} a_K; theta: lam^{-1/2} a_K; phi: c_down a_{K-1} + c_up
// a_{K+1}, the degree-shift form of sin(theta) d/dtheta, for chunk q of K
// tile kt of block (m, parity): the 8 degrees K = m + par + 2 j, j = 64 kt +
// 8 q .. +7.  prep_consts reads the plan's table (before any wait for the
// predecessor); prep_chunk reads alpha and returns the hi parts of the six
// columns (v[0..5]), their lo parts (v[6..11]) and, for m = 1, the u_phi at
// m = 0 column -a_{K,0} (hi v[12], lo v[13]; zero otherwise).  With
// d/dtheta Pt_K^0 = sqrt(K (K+1)) Pt_K^1 (ladder relation, Condon-Shortley
// phase), u_phi at m = 0 is -sum_K alpha_{K,0} Pt_K^1: a sum over the
// order-1 table that needs no division by sin(theta).
__device__ __forceinline__ void prep_consts(const float4* __restrict__ prepc, int N, int m, int par, int kt, int q,
                                            float4 (&cf)[8]) {
    const int ne = ext_even(N, m), n = par ? ext_odd(N, m) : ne;
    const int j0 = kt * TC_TILE_K + q * 8;
    const int r0 = ext_off(N, m) + (par ? ne : 0);
#pragma unroll
    for (int e = 0; e < 8; ++e) cf[e] = (j0 + e < n) ? prepc[r0 + j0 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
}

__device__ __forceinline__ void prep_chunk(const double2* __restrict__ alpha, int N, int m, int par, int kt, int q,
                                           const float4 (&cf)[8], uint4 (&v)[14]) {
    const int ne = ext_even(N, m), n = par ? ext_odd(N, m) : ne;
    const int j0 = kt * TC_TILE_K + q * 8;
    const int lo = m > 0 ? m : 1;
    const int K0 = m + par + 2 * j0;
    const int pk = packed_off(N, m) - lo;   // packed index of degree K is pk + K
    float2 al[17];
#pragma unroll
    for (int e = 0; e < 17; ++e) {
        const int K = K0 - 1 + e;
        double2 x = make_double2(0.0, 0.0);
        if (K >= lo && K <= N) x = alpha[pk + K];
        al[e] = make_float2(f64_to_f32_rn(x.x), f64_to_f32_rn(x.y));
    }
    float c6[6][8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float2 am = al[2 * e], a0 = al[2 * e + 1], ap = al[2 * e + 2];
        c6[0][e] = cf[e].x * a0.x;
        c6[1][e] = cf[e].x * a0.y;
        c6[2][e] = cf[e].y * a0.x;
        c6[3][e] = cf[e].y * a0.y;
        c6[4][e] = fmaf(cf[e].z, am.x, cf[e].w * ap.x);
        c6[5][e] = fmaf(cf[e].z, am.y, cf[e].w * ap.y);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        v[c] = pack_hi(c6[c]);
        v[6 + c] = pack_lo(c6[c]);
    }
    v[12] = v[13] = make_uint4(0u, 0u, 0u, 0u);
    if (m == 1) {
        const double2* a0 = alpha + (packed_off(N, 0) - 1);   // a_{K,0} at a0[K], K = 1 .. N (real)
        float re[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int K = K0 + 2 * e;
            re[e] = (j0 + e < n && K <= N) ? -f64_to_f32_rn(a0[K].x) : 0.f;
        }
        v[12] = pack_hi(re);
        v[13] = pack_lo(re);
    }
}

// The same coefficient sets split over the four lanes (q, p) of a chunk:
// lane p takes the degrees j = 64 kt + 8 q + 2 p, +1 and returns word p (two
// bf16) of each row of the chunk: hi parts w[0..5], lo parts w[6..11], the
// u_phi at m = 0 column (m = 1 only) w[12] (hi), w[13] (lo).
__device__ __forceinline__ void prep_words(const double2* __restrict__ alpha, const float4* __restrict__ prepc, int N,
                                           int m, int par, int kt, int q, int p, uint32_t (&w)[14]) {
    const int ne = ext_even(N, m), n = par ? ext_odd(N, m) : ne;
    const int j0 = kt * TC_TILE_K + q * 8 + 2 * p;
    const int r0 = ext_off(N, m) + (par ? ne : 0);
    const int lo = m > 0 ? m : 1;
    const int K0 = m + par + 2 * j0;          // degree of j0
    const int pk = packed_off(N, m) - lo;     // packed index of degree K is pk + K
    float4 cf[2];
    float2 al[5];                             // degrees K0 - 1 .. K0 + 3
#pragma unroll
    for (int e = 0; e < 2; ++e) cf[e] = (j0 + e < n) ? prepc[r0 + j0 + e] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
    for (int e = 0; e < 5; ++e) {
        const int K = K0 - 1 + e;
        double2 x = make_double2(0.0, 0.0);
        if (K >= lo && K <= N) x = alpha[pk + K];
        al[e] = make_float2(f64_to_f32_rn(x.x), f64_to_f32_rn(x.y));
    }
    float c6[6][2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float2 am = al[2 * e], a0 = al[2 * e + 1], ap = al[2 * e + 2];
        c6[0][e] = cf[e].x * a0.x;
        c6[1][e] = cf[e].x * a0.y;
        c6[2][e] = cf[e].y * a0.x;
        c6[3][e] = cf[e].y * a0.y;
        c6[4][e] = fmaf(cf[e].z, am.x, cf[e].w * ap.x);
        c6[5][e] = fmaf(cf[e].z, am.y, cf[e].w * ap.y);
    }
    auto hi2 = [](float a, float b) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<const uint32_t*>(&h);
    };
    auto lo2 = [](float a, float b) {
        const float la = a - __bfloat162float(__float2bfloat16_rn(a));
        const float lb = b - __bfloat162float(__float2bfloat16_rn(b));
        const __nv_bfloat162 l = __floats2bfloat162_rn(la, lb);
        return *reinterpret_cast<const uint32_t*>(&l);
    };
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        w[c] = hi2(c6[c][0], c6[c][1]);
        w[6 + c] = lo2(c6[c][0], c6[c][1]);
    }
    w[12] = w[13] = 0u;
    if (m == 1) {
        const double2* a0 = alpha + (packed_off(N, 0) - 1);   // a_{K,0} at a0[K], K = 1 .. N (real)
        float re[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const int K = K0 + 2 * e;
            re[e] = (j0 + e < n && K <= N) ? -f64_to_f32_rn(a0[K].x) : 0.f;
        }
        w[12] = hi2(re[0], re[1]);
        w[13] = lo2(re[0], re[1]);
    }
}

// ---------------------------------------------------------------------------
// synthesis
//
// Per order m and parity: g[p][c] = sum_j Pt_{K_j}^m(x_p) b[j][c], the dense
// contraction with A = the transposed table block [nh][pad8(n_par)] (M =
// latitudes, K = degrees, K-major; TMA zero-fills degrees past the block),
// B = the prepacked coefficient tile of the three fields.  Both parities of
// an order go to separate accumulators so that the epilogue forms north =
// E + O, south = E - O directly.

struct TcSynArgs {
    const CUtensorMap* map_hi;   // per (m, parity) block of the transposed tables
    const CUtensorMap* map_lo;
    const int4* items;           // (m, latitude tile, instance group, first K tile of the even | odd
                                 // block << 16), CTA c's list (LPT) at c * istride
    const int* item_cnt;         // items of every CTA
    const unsigned char* btiles; // [group][tile][brows][64] bf16, 128-byte swizzle (k_prep_tc)
    const int* tile_off;         // first tile of block b = 2 m + parity
    float* gsyn;                 // instance i writes gsyn + i * sgs complex entries
    const float* isin;           // 1 / sin(theta_p), FP32
    unsigned* status;
    int N, nh, nlat, nblk, pairs;
    int ng, nb, brows, ntiles, ns;   // instances per group, instances, B rows (= MMA N), tiles, stages
    size_t sgs;
    int istride;                 // item slots per CTA (>= its item count)
    // clusters of CS > 1 CTAs: maps of the same blocks with boxes of 128 / CS latitudes
    const CUtensorMap* map_hi_cs;
    const CUtensorMap* map_lo_cs;
    // SINGLE: the coefficients the builder warps read
    const double2* alpha;
    const float4* prepc;
};

constexpr int TC_SYN_MAXNS = 8;
constexpr int TC_SYN_SMITEMS = 64;   // items per CTA kept in shared memory
constexpr int TC_SYN_BUILDERS = 6;   // warps building coefficient tiles (single-instance synthesis)

__host__ __device__ inline int syn_ndeg(int N, int m, int par) {
    const int n = par ? ext_odd(N, m) : ext_even(N, m);
    return ((n + 7) / 8) * 8;
}
__host__ __device__ inline int syn_nkt(int N, int m, int par) {
    return (syn_ndeg(N, m, par) + TC_TILE_K - 1) / TC_TILE_K;
}
// width of the last K tile of a block, rounded up to the 16-degree MMA chunk
__host__ __device__ inline int syn_tailw(int N, int m, int par) {
    const int rem = syn_ndeg(N, m, par) - (syn_nkt(N, m, par) - 1) * TC_TILE_K;
    return ((rem + 15) / 16) * 16;
}

// Item = (order m, latitude tile of 128 northern nodes, group of ng
// instances): both parities into their own accumulator of brows columns
// (12 per instance: six hi parts, six lo parts of the coefficient sets; then
// two per instance for u_phi at m = 0, filled on order-1 tiles only; hi and
// lo table parts go into the same accumulator, as both multiply the same B
// tile), so one A tile serves every instance of the group.  K chunks of 16
// degrees past the block are skipped.
// NS stages (a compile-time ring keeps the per-stage index arithmetic of the
// single-thread producer and MMA issuer cheap); SINGLE: one instance, 16 B rows.
//
// CS > 1 (batches): the CTAs of a cluster take the same items (m, latitude
// tile) for CS consecutive instance groups (item.z = group / CS).  Each CTA
// loads a slice of 128 / CS latitudes of every table tile and multicasts it
// to the whole cluster, so the table crosses from L2 once per cluster
// instead of once per group; a stage is refilled once the MMAs of every CTA
// of the cluster are done with it (their commits arrive on each CTA's empty
// barrier).
template <int NS, bool SINGLE, int CS = 1>
__global__ void __launch_bounds__(SINGLE ? 192 + 32 * TC_SYN_BUILDERS : 192, 1) k_syn_tc(TcSynArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~uintptr_t(1023));
    constexpr int ns = NS;
    const int brows = SINGLE ? 16 : a.brows;
    const int bbytes = brows * TC_TILE_K * 2;
    unsigned char* A_hi = smem;
    unsigned char* A_lo = A_hi + ns * TC_ATILE;
    unsigned char* Bs = A_lo + ns * TC_ATILE;                    // ns x brows x 128 B
    uint64_t* bars = reinterpret_cast<uint64_t*>(Bs + ns * bbytes);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + ns;
    // accumulator buffers: the single-instance kernel has four (16 columns
    // per parity each), so that an item's epilogue, which waits on global
    // loads and stores, never holds up the MMAs of the items after it
    constexpr int NACC = SINGLE ? 4 : 2;
    uint64_t* acc_full = bars + 2 * ns;
    uint64_t* acc_empty = acc_full + NACC;
    uint64_t* b_full = acc_empty + NACC;                         // SINGLE: coefficient tile of a stage built
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_full + (SINGLE ? ns : 0));
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    // the CTA's first TC_SYN_SMITEMS items, (m, latitude tile, group, first
    // K tile of the even | odd block << 16), read once: every role walks the
    // item list, and dependent global loads per item would stall it
    int4* s_items = reinterpret_cast<int4*>(reinterpret_cast<unsigned char*>(bars) + 512);
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    uint32_t tcols = 32;
    while (tcols < uint32_t(2 * NACC * brows)) tcols <<= 1;
    constexpr uint16_t cmask = uint16_t((1u << CS) - 1u);
    const int crank = CS > 1 ? int(cluster_ctarank()) : 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < ns; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], CS);
            if constexpr (SINGLE) mbar_init(&b_full[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        *abort = 0;
        fence_barrier_init();
    }
    // the lists sit at a fixed stride, so the item loads do not wait on
    // the count (a kernel's first table request waits on this chain)
    const int ib = (blockIdx.x / CS) * a.istride, nI = a.item_cnt[blockIdx.x / CS];
    for (int j = threadIdx.x; j < a.istride && j < TC_SYN_SMITEMS; j += blockDim.x) s_items[j] = a.items[ib + j];
    auto item_meta = [&](int i) -> int4 { return i < TC_SYN_SMITEMS ? s_items[i] : a.items[ib + i]; };
    if (warp == 1) {
        tmem_alloc(tmem_slot, tcols);
        tmem_relinquish();
    }
    tc_fence_before();
    // the cluster's barriers exist before any slice or commit targets them
    if constexpr (CS > 1) cluster_sync();
    else __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int N = a.N, nh = a.nh, nlat = a.nlat;
    pdl_launch();

    if (warp == 0 && SINGLE) {
        if (lane == 0) {
            // the table does not depend on the predecessor (no wait); the
            // builder warps write every stage's coefficient tile. Only the
            // first stage is requested before its data lands: the builders'
            // first coefficient loads would otherwise queue behind every
            // CTA's full pipeline of table requests
            const uint64_t pol = policy_evict_first();
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int4 itm = item_meta(i);
                const int m = itm.x, mt = itm.y;
                for (int par = 0; par < 2; ++par) {
                    const int b = 2 * m + par, nkt = syn_nkt(N, m, par);
                    const int tw = syn_tailw(N, m, par);
                    for (int kt = ((itm.w >> (16 * par)) & 0xFFFF); kt < nkt; ++kt, ++it) {
                        const int s = it % ns;
                        if (it == 1 && !mbar_wait(&a_full[0], 0, abort, a.status)) continue;
                        if (it >= ns && !mbar_wait(&a_empty[s], ((it / ns) - 1) & 1, abort, a.status)) continue;
                        if (*abort) continue;
                        const bool last = kt == nkt - 1;
                        const int w = last ? tw : TC_TILE_K;
                        const int mi = last ? a.nblk + b : b;
                        mbar_arrive_expect_tx(&a_full[s], uint32_t(2 * w * TC_TILE_M * 2));
                        tma_load_2d(A_hi + s * TC_ATILE, &a.map_hi[mi], kt * TC_TILE_K, mt * TC_TILE_M, &a_full[s], pol);
                        tma_load_2d(A_lo + s * TC_ATILE, &a.map_lo[mi], kt * TC_TILE_K, mt * TC_TILE_M, &a_full[s], pol);
                    }
                }
            }
            for (int k = it - ns; k < it; ++k)
                if (k >= 0) mbar_wait(&a_full[k % ns], (k / ns) & 1, abort, a.status);
        }
    } else if (warp == 0) {
        if (lane == 0) {
            // the table tiles of the first ns stages do not depend on the
            // predecessor (the B tiles do): they are requested before the wait,
            // overlapping the coefficient prep, and their B tiles right after it.
            // One group streams the table once (evict-first); several groups
            // re-read it (an ensemble bucket's table: a few MB), so it stays.
            const uint64_t pol = a.nb > a.ng ? policy_evict_last() : policy_evict_first();
            const uint64_t polb = policy_evict_last();
            const unsigned char* pend[NS];
            bool waited = false;
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int4 itm = item_meta(i);
                const int m = itm.x, mt = itm.y, g = itm.z * CS + crank;
                for (int par = 0; par < 2; ++par) {
                    const int b = 2 * m + par, nkt = syn_nkt(N, m, par);
                    const int tw = syn_tailw(N, m, par);
                    const unsigned char* bsrc =
                        a.btiles + (size_t(g) * a.ntiles + size_t(a.tile_off[b])) * size_t(bbytes);
                    for (int kt = ((itm.w >> (16 * par)) & 0xFFFF); kt < nkt; ++kt, ++it) {
                        const int s = it % ns;
                        if (it >= ns) {
                            if (!waited) {
                                pdl_wait();
                                // (an abort may have left a stage without its pend entry)
                                for (int j = 0; j < ns; ++j)
                                    if (!*abort) bulk_g2s(Bs + j * bbytes, pend[j], uint32_t(bbytes), &a_full[j], polb);
                                waited = true;
                            }
                            if (!mbar_wait(&a_empty[s], ((it / ns) - 1) & 1, abort, a.status)) continue;
                        }
                        if (*abort) continue;
                        const bool last = kt == nkt - 1;
                        const int w = last ? tw : TC_TILE_K;
                        const int mi = last ? a.nblk + b : b;
                        mbar_arrive_expect_tx(&a_full[s], uint32_t(2 * w * TC_TILE_M * 2 + bbytes));
                        if constexpr (CS == 1) {
                            tma_load_2d(A_hi + s * TC_ATILE, &a.map_hi[mi], kt * TC_TILE_K, mt * TC_TILE_M, &a_full[s],
                                        pol);
                            tma_load_2d(A_lo + s * TC_ATILE, &a.map_lo[mi], kt * TC_TILE_K, mt * TC_TILE_M, &a_full[s],
                                        pol);
                        } else {
                            // this CTA's slice of latitudes, to every CTA of the cluster
                            constexpr int rows = TC_TILE_M / CS;
                            const int off = crank * rows * 128, y = mt * TC_TILE_M + crank * rows;
                            tma_load_2d_mc(A_hi + s * TC_ATILE + off, &a.map_hi_cs[mi], kt * TC_TILE_K, y, &a_full[s],
                                           cmask, pol);
                            tma_load_2d_mc(A_lo + s * TC_ATILE + off, &a.map_lo_cs[mi], kt * TC_TILE_K, y, &a_full[s],
                                           cmask, pol);
                        }
                        if (waited) bulk_g2s(Bs + s * bbytes, bsrc + size_t(kt) * bbytes, uint32_t(bbytes), &a_full[s], polb);
                        else pend[s] = bsrc + size_t(kt) * bbytes;
                    }
                }
            }
            if (!waited) {
                pdl_wait();
                for (int j = 0; j < it && j < ns; ++j)
                    if (!*abort) bulk_g2s(Bs + j * bbytes, pend[j], uint32_t(bbytes), &a_full[j], polb);
            }
            for (int k = it - ns; k < it; ++k)
                if (k >= 0) mbar_wait(&a_full[k % ns], (k / ns) & 1, abort, a.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(TC_TILE_M, brows);
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int4 itm = item_meta(i);
                const int m = itm.x, mt = itm.y;
                const int buf = i % NACC, use = i / NACC;
                bool ok = true;
                if (i >= NACC) ok = mbar_wait(&acc_empty[buf], (use - 1) & 1, abort, a.status);
                tc_fence_after();
                for (int par = 0; par < 2; ++par) {
                    const int nkt = syn_nkt(N, m, par), nd = syn_ndeg(N, m, par);
                    const int kt0 = (itm.w >> (16 * par)) & 0xFFFF;
                    const uint32_t d = tmem + uint32_t((buf * 2 + par) * brows);
                    for (int kt = kt0; kt < nkt; ++kt, ++it) {
                        const int s = it % ns;
                        bool okA = mbar_wait(&a_full[s], (it / ns) & 1, abort, a.status);
                        if constexpr (SINGLE) okA = okA && mbar_wait(&b_full[s], (it / ns) & 1, abort, a.status);
                        tc_fence_after();
                        // 16-degree chunks of this K tile that hold degrees of the block
                        const int nkk = min(TC_TILE_K, nd - kt * TC_TILE_K + 15) / 16;
                        if (ok && okA && !*abort) {
                            for (int kk = 0; kk < nkk; ++kk) {
                                const uint64_t bd = sdesc_sw128(Bs + s * bbytes + kk * 32);
                                mma_bf16(d, sdesc_sw128(A_hi + s * TC_ATILE + kk * 32), bd, idesc, (kt > kt0) || kk != 0);
                                mma_bf16(d, sdesc_sw128(A_lo + s * TC_ATILE + kk * 32), bd, idesc, 1);
                            }
                        }
                        if constexpr (CS > 1) mma_commit_mc(&a_empty[s], cmask);
                        else mma_commit(&a_empty[s]);
                    }
                }
                mma_commit(&acc_full[buf]);
            }
            if (nI > 0) mbar_wait(&acc_full[(nI - 1) % NACC], ((nI - 1) / NACC) & 1, abort, a.status);
        }
    } else if (warp < 6) {
        pdl_wait();
        const int quarter = warp & 3;
        const size_t ld = size_t(N + 1);
        (void)ld;
        for (int i = 0; i < nI; ++i) {
            const int4 itm = item_meta(i);
            const int m = itm.x, mt = itm.y, g = itm.z * CS + crank, buf = i % NACC;
            const int ngi = SINGLE ? 1 : max(0, min(a.ng, a.nb - g * a.ng));
            // the item's constants are loaded before the wait, so their
            // latency passes while the MMAs run
            const float mm = float(m);
            const int p = mt * TC_TILE_M + quarter * 32 + lane;
            const uint32_t lanes = uint32_t(quarter * 32) << 16;
            const float inv_s = p < nh ? a.isin[p] : 0.f;
            // a parity whose table tiles are all negligible at this latitude
            // tile had no MMA: its accumulator holds no data and counts as 0
            const bool zE = (itm.w & 0xFFFF) >= syn_nkt(N, m, 0);
            const bool zO = (itm.w >> 16) >= syn_nkt(N, m, 1);
            const bool ok = mbar_wait(&acc_full[buf], (i / NACC) & 1, abort, a.status);
            tc_fence_after();
            for (int q = 0; q < ngi; ++q) {
                uint32_t e[12], o[12];
                const uint32_t ce = tmem + lanes + uint32_t((buf * 2 + 0) * brows + 12 * q);
                const uint32_t co = tmem + lanes + uint32_t((buf * 2 + 1) * brows + 12 * q);
                tmem_ld8_nowait(ce, e);
                tmem_ld4_nowait(ce + 8, e + 8);
                tmem_ld8_nowait(co, o);
                tmem_ld4_nowait(co + 8, o + 8);
                // u_phi at m = 0: columns 12 ng + 2 q (hi, lo) of the order-1 item
                uint32_t pe[2], po[2];
                if (m == 1) {   // uniform over the item
                    const uint32_t cp = uint32_t(12 * (SINGLE ? 1 : a.ng) + 2 * q);
                    tmem_ld2_nowait(tmem + lanes + uint32_t((buf * 2 + 0) * brows) + cp, pe);
                    tmem_ld2_nowait(tmem + lanes + uint32_t((buf * 2 + 1) * brows) + cp, po);
                }
                tmem_wait_ld();
                if (!ok || p >= nh || *abort) continue;
                if (m == 1) {
                    const float ev = zE ? 0.f : __uint_as_float(pe[0]) + __uint_as_float(pe[1]);
                    const float ov = zO ? 0.f : __uint_as_float(po[0]) + __uint_as_float(po[1]);
                    float2* o0 = reinterpret_cast<float2*>(a.gsyn) + size_t(g * a.ng + q) * a.sgs;
                    o0[gsyn_index(a.pairs, 2, 0, p, N, nlat)] = make_float2(ev + ov, 0.f);
                    if (nlat - 1 - p != p) o0[gsyn_index(a.pairs, 2, 0, nlat - 1 - p, N, nlat)] = make_float2(ev - ov, 0.f);
                }
                float E[6], O[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) {
                    E[c] = zE ? 0.f : __uint_as_float(e[c]) + __uint_as_float(e[6 + c]);
                    O[c] = zO ? 0.f : __uint_as_float(o[c]) + __uint_as_float(o[6 + c]);
                }
                float2* out = reinterpret_cast<float2*>(a.gsyn) + size_t(g * a.ng + q) * a.sgs;
#pragma unroll
                for (int hemi = 0; hemi < 2; ++hemi) {
                    const int row = hemi == 0 ? p : nlat - 1 - p;
                    if (hemi == 1 && row == p) break;
                    const float sg = hemi == 0 ? 1.f : -1.f;
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        if (f == 2 && m == 0) break;   // written by the order-1 item
                        const float gr = E[2 * f] + sg * O[2 * f];
                        const float gi = E[2 * f + 1] + sg * O[2 * f + 1];
                        float2 ov;
                        if (f == 0) ov = make_float2(gr, gi);
                        else if (f == 1) ov = make_float2(-mm * gi * inv_s, mm * gr * inv_s);
                        else ov = make_float2(-gr * inv_s, -gi * inv_s);
                        out[gsyn_index(a.pairs, f, m, row, N, nlat)] = ov;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);
        }
    } else if constexpr (SINGLE) {
        // builders (warps 6 .. 5 + TC_SYN_BUILDERS): warp 6 + it % TC_SYN_BUILDERS writes stage it's
        // coefficient tile once the stage's slot is free, lane (q, p) word p
        // of chunk q of every row, and announces it on b_full
        // A builder starts on stage it only after its previous stage, it -
        // TC_SYN_BUILDERS, was stored, i.e. after stage it - TC_SYN_BUILDERS
        // - ns was consumed.  Its parity wait for the release of stage it -
        // ns is only unambiguous if stage it - 2 ns was consumed as well,
        // which needs TC_SYN_BUILDERS <= ns.
        static_assert(TC_SYN_BUILDERS <= NS, "builders may not run a full ring ahead");
        const int bw = warp - 6, q = lane >> 2, p = lane & 3;
        bool waited = false;
        int it = 0;
        for (int i = 0; i < nI; ++i) {
            const int4 itm = item_meta(i);
            const int m = itm.x;
            for (int par = 0; par < 2; ++par) {
                const int nkt = syn_nkt(N, m, par);
                for (int kt = ((itm.w >> (16 * par)) & 0xFFFF); kt < nkt; ++kt, ++it) {
                    if (it % TC_SYN_BUILDERS != bw) continue;
                    const int s = it % ns;
                    if (!waited) {
                        pdl_wait();   // alpha may be the predecessor's output
                        waited = true;
                    }
                    // the values first: their loads pass while the slot drains
                    uint32_t w[14];
                    prep_words(a.alpha, a.prepc, N, m, par, kt, q, p, w);
                    if (it >= ns && !mbar_wait(&a_empty[s], ((it / ns) - 1) & 1, abort, a.status)) continue;
                    if (*abort) continue;
                    unsigned char* tile = Bs + s * bbytes;
#pragma unroll
                    for (int r = 0; r < 14; ++r) *reinterpret_cast<uint32_t*>(tile + sw128_chunk(r, q) + 4 * p) = w[r];
                    *reinterpret_cast<uint32_t*>(tile + sw128_chunk(14, q) + 4 * p) = 0u;
                    *reinterpret_cast<uint32_t*>(tile + sw128_chunk(15, q) + 4 * p) = 0u;
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&b_full[s]);
                }
            }
        }
    }
    tc_fence_before();
    // no CTA leaves while another of its cluster may still write its shared memory
    if constexpr (CS > 1) cluster_sync();
    else __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

// B tiles of the batched synthesis: thread (tile, chunk q) of instance
// blockIdx.y stores the chunk's hi parts in rows r0 .. r0+5 and lo parts in
// rows r0+6 .. r0+11, r0 = 12 (instance mod ng), of its group's tile, and on
// order-1 tiles the u_phi at m = 0 column in rows 12 ng + 2 (instance mod
// ng) (hi, lo); rows past the group's instances stay zero.
__global__ void __launch_bounds__(128) k_prep_tc(const double2* __restrict__ alpha, const float4* __restrict__ prepc,
                                                 unsigned char* __restrict__ btiles, const int2* __restrict__ tinfo,
                                                 int ntiles, int N, int n_coeff, int ng, int brows) {
    pdl_launch();
    const int g = blockIdx.x * 16 + (threadIdx.x >> 3), q = threadIdx.x & 7;
    if (g >= ntiles) return;
    const int inst = blockIdx.y;
    alpha += size_t(inst) * n_coeff;
    const int2 ti = tinfo[g];
    const int b = ti.x, kt = ti.y, m = b >> 1, par = b & 1;
    // the plan's table is read before the wait; alpha may be the
    // predecessor's output
    float4 cf[8];
    prep_consts(prepc, N, m, par, kt, q, cf);
    pdl_wait();
    uint4 v[14];
    prep_chunk(alpha, N, m, par, kt, q, cf, v);
    const int grp = inst / ng, row0 = 12 * (inst % ng);
    unsigned char* tile = btiles + (size_t(grp) * ntiles + g) * size_t(brows) * TC_TILE_K * 2;
#pragma unroll
    for (int c = 0; c < 12; ++c) *reinterpret_cast<uint4*>(tile + sw128_chunk(row0 + c, q)) = v[c];
    if (m == 1) {
        const int rp = 12 * ng + 2 * (inst % ng);
        *reinterpret_cast<uint4*>(tile + sw128_chunk(rp, q)) = v[12];
        *reinterpret_cast<uint4*>(tile + sw128_chunk(rp + 1, q)) = v[13];
    }
}

// ---------------------------------------------------------------------------
// host side

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

bool tc_supported(const sphnse_plan* P) { return P->nh % 8 == 0 && P->nh >= 16 && P->nlat % 2 == 0; }

// Tensor maps over the whole [ext row][nh] bf16 tables, the analysis items
// (128-row tiles split into groups of at most 32 / (4 NF) overlapped blocks)
// and their LPT schedule over one CTA per SM.
// max |Pt| of every table row over each 64-latitude chunk (once per plan,
// from the FP64 master table [n_ext][nh])
static const std::vector<float>& tc_chunk_max(sphnse_plan* P) {
    auto& cm = P->tc.chunk_max;
    const int nh = P->nh, nch = (nh + TC_TILE_K - 1) / TC_TILE_K;
    if (cm.size() == size_t(P->n_ext) * nch) return cm;
    cm.assign(size_t(P->n_ext) * nch, 0.f);
    const double* t = P->psyn_host.data();
    for (int r = 0; r < P->n_ext; ++r)
        for (int p = 0; p < nh; ++p) {
            float& v = cm[size_t(r) * nch + p / TC_TILE_K];
            v = std::max(v, float(std::fabs(t[size_t(r) * nh + p])));
        }
    return cm;
}

// first 64-latitude chunk (from the pole) in which one of the rows
// row0 + [s, e) of the given pieces reaches TC_SKIP; at most nch - 1
static int ana_first_chunk(const std::vector<float>& cm, int nch, int row0, const int4* pcs, int np) {
    int c0 = nch - 1;
    for (int j = 0; j < np; ++j)
        for (int r = row0 + pcs[j].z; r < row0 + pcs[j].w; ++r)
            for (int c = 0; c < c0; ++c)
                if (cm[size_t(r) * nch + c] >= TC_SKIP) {
                    c0 = c;
                    break;
                }
    return c0;
}

int tc_setup_analysis(sphnse_plan* P, int nf) {
    if (P->tc.ana_ready && P->tc.ana_nf == nf) return SPHNSE_OK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return SPHNSE_E_UNSUPPORTED;
    auto& T = P->tc;
    for (void* q : {T.map_hi, T.map_lo, static_cast<void*>(T.ana_items), static_cast<void*>(T.ana_off),
                    static_cast<void*>(T.ana_pieces)})
        if (q) cudaFree(q);
    T.map_hi = T.map_lo = nullptr;
    T.ana_items = nullptr;
    T.ana_off = nullptr;
    T.ana_pieces = nullptr;
    T.ana_ready = false;
    T.ana_entries = 0;
    const Tables& t = P->tab[SPHNSE_BF16X3];
    const int N = P->N, nh = P->nh, n_ext = P->n_ext;
    CUtensorMap mh, ml;
    {
        const cuuint64_t dims[2] = {cuuint64_t(nh), cuuint64_t(n_ext)};
        const cuuint64_t strides[1] = {cuuint64_t(nh) * 2};
        const cuuint32_t box[2] = {TC_TILE_K, TC_TILE_M};
        const cuuint32_t es[2] = {1, 1};
        for (int lo = 0; lo < 2; ++lo) {
            CUresult r = enc(lo ? &ml : &mh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(lo ? t.syn_lo : t.syn),
                             dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return SPHNSE_E_CUDA;
        }
    }
    // pieces of every tile: the blocks (m, parity) overlapping rows [128 T, 128 T + 128)
    const int maxp = TC_ANA_BROWS / (4 * nf);
    const int ntile = (n_ext + TC_TILE_M - 1) / TC_TILE_M;
    std::vector<int4> pieces, items;
    std::vector<double> cost;
    {
        std::vector<std::vector<int4>> per(ntile);
        for (int m = 0; m <= N; ++m)
            for (int par = 0; par < 2; ++par) {
                const int ne = ext_even(N, m);
                const int r0 = ext_off(N, m) + (par ? ne : 0), nr = par ? ext_odd(N, m) : ne;
                for (int r = r0; r < r0 + nr;) {
                    const int tt = r / TC_TILE_M, end = std::min(r0 + nr, (tt + 1) * TC_TILE_M);
                    per[tt].push_back(make_int4(m, par, r - tt * TC_TILE_M, end - tt * TC_TILE_M));
                    r = end;
                }
            }
        const auto& cm = tc_chunk_max(P);
        const int nch = (nh + TC_TILE_K - 1) / TC_TILE_K;
        for (int tt = 0; tt < ntile; ++tt)
            for (size_t j0 = 0; j0 < per[tt].size(); j0 += maxp) {
                const int np = int(std::min<size_t>(maxp, per[tt].size() - j0));
                const int ncol = ((4 * nf * np + 15) / 16) * 16;
                const int kt0 = ana_first_chunk(cm, nch, tt * TC_TILE_M, per[tt].data() + j0, np);
                items.push_back(make_int4(tt * TC_TILE_M, int(pieces.size()), np, ncol | (kt0 << 16)));
                for (size_t j = j0; j < j0 + np; ++j)
                    T.ana_entries += double(per[tt][j].w - per[tt][j].z) * (nh - std::min(nh, kt0 * TC_TILE_K));
                int rows = 0;
                for (int j = 0; j < np; ++j) {
                    pieces.push_back(per[tt][j0 + j]);
                    rows += per[tt][j0 + j].w - per[tt][j0 + j].z;
                }
                cost.push_back((TC_TILE_M + 24 * np) * double(nch - kt0) / nch);
                (void)rows;
            }
    }
    // LPT: largest items first onto the least-loaded CTA
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    const int G = std::min<int>(P->n_cta, int(items.size()));
    std::vector<std::vector<int4>> bins(G);
    std::vector<double> load(G, 0.0);
    for (int idx : order) {
        int b = int(std::min_element(load.begin(), load.end()) - load.begin());
        bins[b].push_back(items[idx]);
        load[b] += cost[idx];
    }
    std::vector<int4> flat;
    std::vector<int> off(1, 0);
    for (auto& bi : bins) {
        flat.insert(flat.end(), bi.begin(), bi.end());
        off.push_back(int(flat.size()));
    }
    if (cudaMalloc(&T.map_hi, sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(&T.map_lo, sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.ana_items), flat.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.ana_off), off.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.ana_pieces), pieces.size() * sizeof(int4)) != cudaSuccess)
        return SPHNSE_E_NOMEM;
    cudaMemcpy(T.map_hi, &mh, sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    cudaMemcpy(T.map_lo, &ml, sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    cudaMemcpy(T.ana_items, flat.data(), flat.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(T.ana_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(T.ana_pieces, pieces.data(), pieces.size() * sizeof(int4), cudaMemcpyHostToDevice);
    T.ana_cta = G;
    T.ana_nf = nf;
    T.ana_ready = true;
    return check_cuda(cudaGetLastError());
}

template <int NF>
static int ana_tc_t(sphnse_plan* P) {
    const int nkt = (P->nh + TC_TILE_K - 1) / TC_TILE_K;
    const size_t sm = 1024 + 2 * size_t(TC_ANA_NS) * TC_ATILE + 2 * size_t(nkt) * TC_ANA_BTILE + 256;
    if (sm > 227 * 1024) return SPHNSE_E_UNSUPPORTED;
    allow_dynamic_smem(reinterpret_cast<const void*>(k_ana_tc<NF>), sm);
    TcAnaArgs a{reinterpret_cast<const CUtensorMap*>(P->tc.map_hi), reinterpret_cast<const CUtensorMap*>(P->tc.map_lo),
                P->tc.ana_items, P->tc.ana_off, P->tc.ana_pieces,
                reinterpret_cast<const float*>(P->d_gana), reinterpret_cast<float*>(P->d_hana), P->d_status,
                P->N, P->nh, P->nlat, nkt, P->n_ext};
    stage_begin(P, SPHNSE_STAGE_ANALYSIS);
    const cudaError_t e = launch_pdl(k_ana_tc<NF>, dim3(P->tc.ana_cta), dim3(320), sm, P->stream, a);
    stage_end(P, SPHNSE_STAGE_ANALYSIS);
    return check_cuda(e);
}

int launch_analysis_tc(sphnse_plan* P, int nfields) {
    int rc = tc_setup_analysis(P, nfields);
    if (rc) return rc;
    return nfields == 3 ? ana_tc_t<3>(P) : ana_tc_t<2>(P);
}

// Order groups of the fused analysis: consecutive orders whose rows (at
// most two orders' worth) go through consecutive 128-row tiles, each tile
// with at most two orders (four blocks: the pieces a tile holds).  Each CTA
// takes whole groups, LPT by the table tiles they read.
static int tc_setup_analysis_fin(sphnse_plan* P) {
    auto& T = P->tc;
    if (T.anf_ready) return SPHNSE_OK;
    int rc = tc_setup_analysis(P, 2);
    if (rc) return rc;
    const int N = P->N, nh = P->nh;
    const auto& cm = tc_chunk_max(P);
    const int nch = (nh + TC_TILE_K - 1) / TC_TILE_K;
    struct Group {
        std::vector<int4> items, og;
        std::vector<std::vector<int4>> pcs;
        double cost = 0;
    };
    std::vector<Group> groups;
    double entries = 0;
    // a group takes the next order while its rows fit a stage buffer, every
    // 128-row tile still holds at most two orders (four blocks), and the
    // merge saves a tile
    const int cap = std::max(2 * (N + 2), TC_TILE_M);
    auto ntiles = [](int rows) { return (rows + TC_TILE_M - 1) / TC_TILE_M; };
    auto two_per_tile = [&](int m, int m1) {
        const int r0 = ext_off(N, m), r1 = ext_off(N, m1);
        for (int t = r0; t < r1; t += TC_TILE_M) {
            const int te = std::min(r1, t + TC_TILE_M);
            int k = 0;
            for (int mm = m; mm < m1; ++mm)
                if (ext_off(N, mm) < te && ext_off(N, mm + 1) > t) ++k;
            if (k > 2) return false;
        }
        return true;
    };
    for (int m = 0; m <= N;) {
        int m1 = m + 1;
        while (m1 <= N && ext_off(N, m1 + 1) - ext_off(N, m) <= cap && two_per_tile(m, m1 + 1) &&
               ntiles(ext_off(N, m1 + 1) - ext_off(N, m)) <
                   ntiles(ext_off(N, m1) - ext_off(N, m)) + ntiles(ext_count(N, m1)))
            ++m1;
        const int row0 = ext_off(N, m), rows = ext_off(N, m1) - row0;
        Group g;
        for (int t0 = 0; t0 < rows; t0 += TC_TILE_M) {
            const int r0 = row0 + t0, r1 = row0 + std::min(rows, t0 + TC_TILE_M);
            std::vector<int4> pc;
            for (int mm = m; mm < m1; ++mm)
                for (int par = 0; par < 2; ++par) {
                    const int ne = ext_even(N, mm);
                    const int b0 = ext_off(N, mm) + (par ? ne : 0), b1 = b0 + (par ? ext_odd(N, mm) : ne);
                    const int s0 = std::max(b0, r0), s1 = std::min(b1, r1);
                    if (s0 < s1) pc.push_back(make_int4(mm, par, s0 - r0, s1 - r0));
                }
            const int np = int(pc.size());
            const int ncol = ((8 * np + 15) / 16) * 16;
            const int kt0 = ana_first_chunk(cm, nch, r0, pc.data(), np);
            for (const int4& q : pc) entries += double(q.w - q.z) * (nh - std::min(nh, kt0 * TC_TILE_K));
            const int bj = (r1 - r0 + 15) / 16 - 1;
            g.items.push_back(make_int4(r0, 0, np, ncol | (kt0 << 16) | (bj << 24)));
            g.og.push_back(make_int4(row0, m, m1, r1 == row0 + rows ? 1 : 0));
            g.pcs.push_back(pc);
            // a CTA's time follows its K-tile stages (eight MMAs each)
            g.cost += double(nch - kt0);
        }
        groups.push_back(std::move(g));
        m = m1;
    }
    std::vector<int> order(groups.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return groups[x].cost > groups[y].cost; });
    const int G = std::min<int>(P->n_cta, int(groups.size()));
    std::vector<std::vector<int>> bins(G);
    std::vector<double> load(G, 0.0);
    for (int idx : order) {
        const int b = int(std::min_element(load.begin(), load.end()) - load.begin());
        bins[b].push_back(idx);
        load[b] += groups[idx].cost;
    }
    // maps with boxes of 16 .. 128 rows: a group's last tile reads its own rows
    // rounded up to 16, not a full tile of the next group's
    EncodeTiledFn enc = encode_fn();
    if (!enc) return SPHNSE_E_UNSUPPORTED;
    CUtensorMap mh[8], ml[8];
    {
        const Tables& t = P->tab[SPHNSE_BF16X3];
        const cuuint64_t dims[2] = {cuuint64_t(nh), cuuint64_t(P->n_ext)};
        const cuuint64_t strides[1] = {cuuint64_t(nh) * 2};
        const cuuint32_t es[2] = {1, 1};
        for (int j = 0; j < 8; ++j) {
            const cuuint32_t box[2] = {TC_TILE_K, cuuint32_t(16 * (j + 1))};
            for (int lo = 0; lo < 2; ++lo) {
                CUresult r = enc(lo ? &ml[j] : &mh[j], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                 const_cast<void*>(lo ? t.syn_lo : t.syn), dims, strides, box, es,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) return SPHNSE_E_CUDA;
            }
        }
    }
    std::vector<int4> items, og, pieces;
    std::vector<int> off(1, 0);
    for (auto& bi : bins) {
        for (int gi : bi) {
            const Group& g = groups[gi];
            for (size_t k = 0; k < g.items.size(); ++k) {
                int4 it = g.items[k];
                it.y = int(pieces.size());
                pieces.insert(pieces.end(), g.pcs[k].begin(), g.pcs[k].end());
                items.push_back(it);
                og.push_back(g.og[k]);
            }
        }
        off.push_back(int(items.size()));
    }
    if (cudaMalloc(&T.anf_map_hi, sizeof(mh)) != cudaSuccess || cudaMalloc(&T.anf_map_lo, sizeof(ml)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.anf_items), items.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.anf_og), og.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.anf_off), off.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.anf_pieces), pieces.size() * sizeof(int4)) != cudaSuccess)
        return SPHNSE_E_NOMEM;
    cudaMemcpy(T.anf_map_hi, mh, sizeof(mh), cudaMemcpyHostToDevice);
    cudaMemcpy(T.anf_map_lo, ml, sizeof(ml), cudaMemcpyHostToDevice);
    cudaMemcpy(T.anf_items, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(T.anf_og, og.data(), og.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(T.anf_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(T.anf_pieces, pieces.data(), pieces.size() * sizeof(int4), cudaMemcpyHostToDevice);
    T.anf_cta = G;
    T.ana_entries = entries;
    T.anf_ready = true;
    return check_cuda(cudaGetLastError());
}

bool tc_rhs_fused(sphnse_plan* P) {
    if (P->precision != SPHNSE_BF16X3 || !tc_supported(P) || !ring4_ok(P)) return false;
    if (tc_setup_synthesis(P) || tc_setup_analysis_fin(P)) return false;
    const TcBatch& B = P->tc.single;
    if (!(B.nb == 1 && B.ng == 1 && B.brows == 16 && B.ns == 6 && B.cs == 1)) return false;
    const int nkt = (P->nh + TC_TILE_K - 1) / TC_TILE_K;
    const int srows = std::max(2 * (P->N + 2), TC_TILE_M);
    const size_t sm = 1024 + 2 * size_t(TC_ANA_NS_FIN) * TC_ATILE + 2 * size_t(nkt) * TC_ANA_BTILE + 256 +
                      2 * size_t(srows) * 4 * sizeof(float);
    return sm <= 227 * 1024;
}

int launch_analysis_finish_tc(sphnse_plan* P, const double* alpha, const double* forcing, double* out) {
    int rc = tc_setup_analysis_fin(P);
    if (rc) return rc;
    const int nkt = (P->nh + TC_TILE_K - 1) / TC_TILE_K;
    // stages, B tiles, barriers (256 B) and two stage buffers of an order
    // group's rows (at most two orders, 2 (N + 2) rows)
    const int srows = std::max(2 * (P->N + 2), TC_TILE_M);
    const size_t sm = 1024 + 2 * size_t(TC_ANA_NS_FIN) * TC_ATILE + 2 * size_t(nkt) * TC_ANA_BTILE + 256 +
                      2 * size_t(srows) * 4 * sizeof(float);
    if (sm > 227 * 1024) return SPHNSE_E_UNSUPPORTED;
    allow_dynamic_smem(reinterpret_cast<const void*>(k_ana_tc<2, true>), sm);
    TcAnaArgs a{reinterpret_cast<const CUtensorMap*>(P->tc.anf_map_hi),
                reinterpret_cast<const CUtensorMap*>(P->tc.anf_map_lo), P->tc.anf_items, P->tc.anf_off,
                P->tc.anf_pieces,
                reinterpret_cast<const float*>(P->d_gana), nullptr, P->d_status,
                P->N, P->nh, P->nlat, nkt, P->n_ext,
                P->tc.anf_og, reinterpret_cast<const double2*>(alpha), reinterpret_cast<const double2*>(forcing),
                reinterpret_cast<double2*>(out), P->d_finc32, P->nu, P->coriolis_split ? P->Omega : 0.0, srows,
                P->done_cnt, P->done_flag, P->done_ticket};
    stage_begin(P, SPHNSE_STAGE_ANALYSIS);
    const cudaError_t e = launch_pdl(k_ana_tc<2, true>, dim3(P->tc.anf_cta), dim3(448), sm, P->stream, a);
    stage_end(P, SPHNSE_STAGE_ANALYSIS);
    return check_cuda(e);
}

// Transposed, padded bf16 hi/lo tables for the synthesis (block (m, parity)
// stored [nh][pad8(n_par)]) and their tensor maps.
// Tensor maps of every (m, parity) block of the transposed tables with
// boxes of `rows` latitudes: entries [0, nblk) box 64 degrees for full K
// tiles, [nblk, 2 nblk) box syn_tailw for the last K tile (a narrower box
// keeps the 128-byte row pitch of the swizzled tile, so the MMA descriptors
// are the same and only the 16-degree chunks it fills are read).
static int syn_maps(sphnse_plan* P, int rows, void** dhi, void** dlo) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return SPHNSE_E_UNSUPPORTED;
    const auto& T = P->tc;
    const int N = P->N, nh = P->nh, nblk = 2 * (N + 1);
    std::vector<CUtensorMap> mh(2 * nblk), ml(2 * nblk);
    for (int b = 0; b < nblk; ++b) {
        const int m = b / 2, par = b % 2;
        const int np = syn_ndeg(N, m, par);
        const cuuint64_t dims[2] = {cuuint64_t(np), cuuint64_t(nh)};
        const cuuint64_t strides[1] = {cuuint64_t(np) * 2};
        const cuuint32_t es[2] = {1, 1};
        for (int tail = 0; tail < 2; ++tail) {
            const cuuint32_t box[2] = {cuuint32_t(tail ? syn_tailw(N, m, par) : TC_TILE_K), cuuint32_t(rows)};
            for (int l = 0; l < 2; ++l) {
                __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(l ? T.tsyn_lo : T.tsyn_hi) + T.tsyn_off[b];
                CUresult r = enc(l ? &ml[tail * nblk + b] : &mh[tail * nblk + b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                                 base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                 CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                 CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) return SPHNSE_E_CUDA;
            }
        }
    }
    if (cudaMalloc(dhi, 2 * nblk * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(dlo, 2 * nblk * sizeof(CUtensorMap)) != cudaSuccess)
        return SPHNSE_E_NOMEM;
    cudaMemcpy(*dhi, mh.data(), 2 * nblk * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    cudaMemcpy(*dlo, ml.data(), 2 * nblk * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    return SPHNSE_OK;
}

int tc_setup_synthesis(sphnse_plan* P) {
    if (P->tc.syn_ready) return SPHNSE_OK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return SPHNSE_E_UNSUPPORTED;
    int rc_maps;
    const int N = P->N, nh = P->nh;
    const int nblk = 2 * (N + 1);
    std::vector<size_t> off(nblk + 1, 0);
    for (int m = 0; m <= N; ++m)
        for (int par = 0; par < 2; ++par) {
            const int n = par ? ext_odd(N, m) : ext_even(N, m);
            off[2 * m + par + 1] = off[2 * m + par] + size_t(nh) * ((n + 7) / 8) * 8;
        }
    const size_t total = off[nblk];
    std::vector<__nv_bfloat16> hi(total, __float2bfloat16_rn(0.f)), lo(total, __float2bfloat16_rn(0.f));
    const double* src = P->psyn_host.data();
    for (int m = 0; m <= N; ++m)
        for (int par = 0; par < 2; ++par) {
            const int ne = ext_even(N, m);
            const int n = par ? ext_odd(N, m) : ne;
            const int np = ((n + 7) / 8) * 8;
            const int r0 = ext_off(N, m) + (par ? ne : 0);
            const size_t o = off[2 * m + par];
            for (int j = 0; j < n; ++j)
                for (int p = 0; p < nh; ++p) {
                    const double v = src[size_t(r0 + j) * nh + p];
                    const __nv_bfloat16 h = __float2bfloat16_rn(float(v));
                    hi[o + size_t(p) * np + j] = h;
                    lo[o + size_t(p) * np + j] = __float2bfloat16_rn(float(v - double(__bfloat162float(h))));
                }
        }
    auto& T = P->tc;
    if (cudaMalloc(&T.tsyn_hi, total * 2) != cudaSuccess || cudaMalloc(&T.tsyn_lo, total * 2) != cudaSuccess)
        return SPHNSE_E_NOMEM;
    cudaMemcpy(T.tsyn_hi, hi.data(), total * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(T.tsyn_lo, lo.data(), total * 2, cudaMemcpyHostToDevice);
    T.tsyn_off.assign(off.begin(), off.end());
    if ((rc_maps = syn_maps(P, TC_TILE_M, &T.smap_hi, &T.smap_lo))) return rc_maps;
    // tile list of the B operand: one tile per (m, parity, K tile)
    std::vector<int> toff(nblk + 1, 0);
    for (int b = 0; b < nblk; ++b) toff[b + 1] = toff[b] + syn_nkt(N, b / 2, b % 2);
    if (cudaMalloc(reinterpret_cast<void**>(&T.tile_off), toff.size() * sizeof(int)) != cudaSuccess)
        return SPHNSE_E_NOMEM;
    cudaMemcpy(T.tile_off, toff.data(), toff.size() * sizeof(int), cudaMemcpyHostToDevice);
    {   // flat tile list (block, K tile) for k_prep_tc
        std::vector<int2> ti;
        for (int b = 0; b < nblk; ++b)
            for (int kt = 0; kt < toff[b + 1] - toff[b]; ++kt) ti.push_back(make_int2(b, kt));
        if (cudaMalloc(reinterpret_cast<void**>(&T.tile_info), ti.size() * sizeof(int2)) != cudaSuccess)
            return SPHNSE_E_NOMEM;
        cudaMemcpy(T.tile_info, ti.data(), ti.size() * sizeof(int2), cudaMemcpyHostToDevice);
        T.ntiles = int(ti.size());
    }
    T.syn_entries = 0;
    {   // first significant K tile of every (block, latitude tile)
        const auto& cm = tc_chunk_max(P);
        const int nch = (nh + TC_TILE_K - 1) / TC_TILE_K, nmt = (nh + TC_TILE_M - 1) / TC_TILE_M;
        std::vector<int> k0(size_t(nblk) * nmt);
        for (int b = 0; b < nblk; ++b) {
            const int m = b / 2, par = b % 2;
            const int n = par ? ext_odd(N, m) : ext_even(N, m);
            const int r0 = ext_off(N, m) + (par ? ext_even(N, m) : 0), nkt = syn_nkt(N, m, par);
            for (int mt = 0; mt < nmt; ++mt) {
                int kt0 = nkt;   // nkt: the whole block is negligible on this latitude tile
                for (int j = 0; j < n && j / TC_TILE_K < kt0; ++j) {
                    const size_t r = size_t(r0 + j) * nch;
                    float v = cm[r + 2 * mt];
                    if (2 * mt + 1 < nch) v = std::max(v, cm[r + 2 * mt + 1]);
                    if (v >= TC_SKIP) kt0 = std::min(kt0, j / TC_TILE_K);
                }
                k0[size_t(b) * nmt + mt] = kt0;
                const int rows = std::min(nh, (mt + 1) * TC_TILE_M) - mt * TC_TILE_M;
                for (int kt = kt0; kt < nkt; ++kt)
                    T.syn_entries += double(rows) * std::min(TC_TILE_K, n - kt * TC_TILE_K);
            }
        }
        T.syn_kt0_host = k0;   // the item lists carry it (tc_batch_init)
    }
    T.tsyn_bytes = 2 * total * 2;
    T.syn_ready = true;
    const int rc = tc_batch_init(P, 1, &T.single);
    if (rc) return rc;
    return check_cuda(cudaGetLastError());
}

static int syn_cluster_capacity(int ns, int cs, size_t smem);

// Instance groups of a batch of nb instances of one truncation: ng <= 9
// instances share every A tile (MMA N = brows = 14 ng rounded up to 16),
// B tiles [group][tile][brows][64], items (m, latitude tile, group) in LPT
// order over one CTA per SM.  cs > 1: clusters of cs CTAs take the items
// of cs consecutive groups together (item.z = group / cs, the group count
// a multiple of cs) and share every table tile by multicast; the schedule
// has one bin per cluster that can be resident at once.
int tc_batch_init(sphnse_plan* P, int nb, TcBatch* B, int ngmax, int nsmax, int cs) {
    if (nb < 1 || ngmax < 1 || nsmax < 1 || (cs != 1 && cs != 2 && cs != 4)) return SPHNSE_E_ARG;
    const int N = P->N, nh = P->nh;
    TcBatch T;
    T.nb = nb;
    T.cs = cs;
    // 14 B rows per instance (12 coefficient rows, 2 for u_phi at m = 0); two
    // accumulators of brows <= 128 columns per buffer fit TMEM's 512
    T.ng = std::min(nb, std::min(ngmax, 9));
    T.ngroups = (nb + T.ng - 1) / T.ng;
    T.ngroups = ((T.ngroups + cs - 1) / cs) * cs;
    T.ng = (nb + T.ngroups - 1) / T.ngroups;   // balanced groups
    T.brows = ((14 * T.ng + 15) / 16) * 16;
    const size_t stage = 2 * size_t(TC_ATILE) + size_t(T.brows) * TC_TILE_K * 2;
    T.ns = int(std::min<size_t>(std::min(nsmax, 6), (size_t(227) * 1024 - 1024 - 512 - TC_SYN_SMITEMS * sizeof(int4)) / stage));
    if (cs > 1) {
        // slice maps (128 / cs latitudes per box) of this plan, once
        void** hi = cs == 2 ? &P->tc.smap_hi_c2 : &P->tc.smap_hi_c4;
        void** lo = cs == 2 ? &P->tc.smap_lo_c2 : &P->tc.smap_lo_c4;
        if (!*hi) {
            const int rc = syn_maps(P, TC_TILE_M / cs, hi, lo);
            if (rc) return rc;
        }
    }
    const size_t bytes = size_t(T.ngroups) * P->tc.ntiles * T.brows * TC_TILE_K * 2;
    if (cudaMalloc(reinterpret_cast<void**>(&T.btiles), bytes) != cudaSuccess) return SPHNSE_E_NOMEM;
    cudaMemset(T.btiles, 0, bytes);
    const int nmt = (nh + TC_TILE_M - 1) / TC_TILE_M;
    std::vector<int4> its;
    std::vector<double> cost;
    for (int gq = 0; gq < T.ngroups / cs; ++gq) {
        const int ngi = std::max(0, std::min(T.ng, nb - gq * cs * T.ng));
        for (int m = 0; m <= N; ++m)
            for (int mt = 0; mt < nmt; ++mt) {
                const auto& k0 = P->tc.syn_kt0_host;
                const int k0e = k0[size_t(2 * m) * nmt + mt], k0o = k0[size_t(2 * m + 1) * nmt + mt];
                its.push_back(make_int4(m, mt, gq, k0e | (k0o << 16)));
                // streamed stages (A and B bytes) plus a fixed cost per item and the epilogue of the group
                const int nst = syn_nkt(N, m, 0) - k0e + syn_nkt(N, m, 1) - k0o;
                cost.push_back(nst * (1.0 + T.brows / 256.0) + 1.0 + 0.1 * (ngi - 1));
            }
    }
    std::vector<int> order(its.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    int bins_max = P->n_cta;
    if (cs > 1) {
        const size_t sm = 1024 + size_t(T.ns) * (2 * size_t(TC_ATILE) + size_t(T.brows) * TC_TILE_K * 2) + 512;
        bins_max = syn_cluster_capacity(T.ns, cs, sm);
        if (bins_max < 1) {
            tc_batch_free(&T);
            return SPHNSE_E_UNSUPPORTED;
        }
    }
    const int G = std::min<int>(bins_max, int(its.size()));
    std::vector<std::vector<int4>> bins(G);
    std::vector<double> load(G, 0.0);
    for (int idx : order) {
        const int bb = int(std::min_element(load.begin(), load.end()) - load.begin());
        bins[bb].push_back(its[idx]);
        load[bb] += cost[idx];
    }
    // within a CTA, long and short items alternate (LPT leaves the short
    // ones last, where their epilogues and new tensor maps, not the table
    // stream, would set the pace)
    for (auto& bi : bins) {
        std::vector<int4> alt;
        alt.reserve(bi.size());
        for (size_t lo = 0, hi = bi.size(); lo < hi;) {
            alt.push_back(bi[lo++]);
            if (lo < hi) alt.push_back(bi[--hi]);
        }
        bi.swap(alt);
    }
    // every CTA's list at a fixed stride (padded with unused slots)
    size_t stride = 1;
    for (auto& bi : bins) stride = std::max(stride, bi.size());
    std::vector<int4> flat(size_t(G) * stride, make_int4(0, 0, 0, 0));
    std::vector<int> cnt(G);
    for (int bb = 0; bb < G; ++bb) {
        std::copy(bins[bb].begin(), bins[bb].end(), flat.begin() + size_t(bb) * stride);
        cnt[bb] = int(bins[bb].size());
    }
    if (cudaMalloc(reinterpret_cast<void**>(&T.items), flat.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.cnt), cnt.size() * sizeof(int)) != cudaSuccess) {
        tc_batch_free(&T);
        return SPHNSE_E_NOMEM;
    }
    cudaMemcpy(T.items, flat.data(), flat.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(T.cnt, cnt.data(), cnt.size() * sizeof(int), cudaMemcpyHostToDevice);
    T.istride = int(stride);
    T.ncta = G * cs;
    *B = T;
    return check_cuda(cudaGetLastError());
}

void tc_batch_free(TcBatch* B) {
    for (void* q : {static_cast<void*>(B->btiles), static_cast<void*>(B->items), static_cast<void*>(B->cnt)})
        if (q) cudaFree(q);
    *B = TcBatch();
}

int launch_prep_tc_batch(sphnse_plan* P, const TcBatch& B, const double* alpha) {
    stage_begin(P, SPHNSE_STAGE_PREP);
    const cudaError_t e = launch_pdl(k_prep_tc, dim3((P->tc.ntiles + 15) / 16, B.nb), dim3(128), 0, P->stream,
                                     reinterpret_cast<const double2*>(alpha), static_cast<const float4*>(P->d_prepc32),
                                     B.btiles, static_cast<const int2*>(P->tc.tile_info), P->tc.ntiles, P->N,
                                     P->n_coeff, B.ng, B.brows);
    stage_end(P, SPHNSE_STAGE_PREP);
    return check_cuda(e);
}

typedef void (*SynKernel)(TcSynArgs);

static SynKernel syn_kernel(int ns, bool single, int cs) {
    if (single) return ns == 6 && cs == 1 ? k_syn_tc<6, true> : nullptr;
    if (cs == 1) return ns == 6 ? k_syn_tc<6, false> : ns == 5 ? k_syn_tc<5, false> : ns == 4 ? k_syn_tc<4, false>
                                                                                               : nullptr;
    if (cs == 2) return ns == 6 ? k_syn_tc<6, false, 2> : ns == 5 ? k_syn_tc<5, false, 2> : ns == 4 ? k_syn_tc<4, false, 2>
                                                                                                     : nullptr;
    if (cs == 4) return ns == 6 ? k_syn_tc<6, false, 4> : ns == 5 ? k_syn_tc<5, false, 4> : ns == 4 ? k_syn_tc<4, false, 4>
                                                                                                     : nullptr;
    return nullptr;
}

// Clusters of cs CTAs (smem bytes each) that can be resident at once.
static int syn_cluster_capacity(int ns, int cs, size_t smem) {
    SynKernel kern = syn_kernel(ns, false, cs);
    if (!kern || smem > 227 * 1024) return 0;
    allow_dynamic_smem(reinterpret_cast<const void*>(kern), smem);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cs);
    cfg.blockDim = dim3(192);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

int launch_synthesis_tc_batch(sphnse_plan* P, const TcBatch& B, float* gsyn, size_t sg_floats, int pairs,
                              const double* alpha) {
    // 1 KB alignment slack, the stages, 512 B of barriers, the item table
    const size_t sm = 1024 + size_t(B.ns) * (2 * size_t(TC_ATILE) + size_t(B.brows) * TC_TILE_K * 2) + 512 +
                      TC_SYN_SMITEMS * sizeof(int4);
    if (sm > 227 * 1024 || B.ns > TC_SYN_MAXNS) return SPHNSE_E_UNSUPPORTED;
    // one instance with alpha given: the kernel builds its coefficient tiles
    const bool single = alpha && B.nb == 1 && B.ng == 1 && B.brows == 16 && B.ns == 6 && B.cs == 1;
    SynKernel kern = syn_kernel(B.ns, single, B.cs);
    if (!kern) return SPHNSE_E_UNSUPPORTED;
    allow_dynamic_smem(reinterpret_cast<const void*>(kern), sm);
    const auto& T = P->tc;
    TcSynArgs a{reinterpret_cast<const CUtensorMap*>(T.smap_hi), reinterpret_cast<const CUtensorMap*>(T.smap_lo),
                B.items, B.cnt, B.btiles, T.tile_off, gsyn,
                P->d_isin32, P->d_status, P->N, P->nh, P->nlat, 2 * (P->N + 1), pairs,
                B.ng, B.nb, B.brows, T.ntiles, B.ns, sg_floats / 2, B.istride,
                reinterpret_cast<const CUtensorMap*>(B.cs == 2 ? T.smap_hi_c2 : T.smap_hi_c4),
                reinterpret_cast<const CUtensorMap*>(B.cs == 2 ? T.smap_lo_c2 : T.smap_lo_c4),
                reinterpret_cast<const double2*>(alpha), P->d_prepc32};
    const int threads = single ? 192 + 32 * TC_SYN_BUILDERS : 192;
    stage_begin(P, SPHNSE_STAGE_SYNTHESIS);
    cudaError_t e;
    if (B.cs == 1) {
        e = launch_pdl(kern, dim3(B.ncta), dim3(threads), sm, P->stream, a);
    } else {
        prefer_max_smem(reinterpret_cast<const void*>(kern));
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(B.ncta);
        cfg.blockDim = dim3(threads);
        cfg.dynamicSmemBytes = sm;
        cfg.stream = P->stream;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = B.cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        e = cudaLaunchKernelEx(&cfg, kern, a);
    }
    stage_end(P, SPHNSE_STAGE_SYNTHESIS);
    return check_cuda(e);
}

// The plan's own instance: the synthesis builds its coefficient tiles from
// alpha itself (no prep kernel, one launch boundary fewer per RHS); a batch
// shape other than the single one takes the prep kernel's tiles.
int launch_synthesis_tc(sphnse_plan* P, const double* alpha, int pairs) {
    int rc = tc_setup_synthesis(P);
    if (rc) return rc;
    const TcBatch& B = P->tc.single;
    if (!(B.nb == 1 && B.ng == 1 && B.brows == 16 && B.ns == 6 && B.cs == 1)) {
        if ((rc = launch_prep_tc_batch(P, B, alpha))) return rc;
        alpha = nullptr;
    }
    return launch_synthesis_tc_batch(P, B, reinterpret_cast<float*>(P->d_gsyn), 0, pairs, alpha);
}

// pieces of every 128-row tile of the [ext row] table: the blocks (m, parity)
// overlapping rows [128 T, 128 T + 128), with their tile-row range
static std::vector<std::vector<int4>> tile_pieces(int N, int n_ext) {
    const int ntile = (n_ext + TC_TILE_M - 1) / TC_TILE_M;
    std::vector<std::vector<int4>> per(ntile);
    for (int m = 0; m <= N; ++m)
        for (int par = 0; par < 2; ++par) {
            const int ne = ext_even(N, m);
            const int r0 = ext_off(N, m) + (par ? ne : 0), nr = par ? ext_odd(N, m) : ne;
            for (int r = r0; r < r0 + nr;) {
                const int tt = r / TC_TILE_M, end = std::min(r0 + nr, (tt + 1) * TC_TILE_M);
                per[tt].push_back(make_int4(m, par, r - tt * TC_TILE_M, end - tt * TC_TILE_M));
                r = end;
            }
        }
    return per;
}

// Batched analysis of nb instances (NF = 2): items (tile, <= 32 slots of
// (block, instance)), LPT over one CTA per SM, and the S-tile buffer.
int tc_batch_ana_init(sphnse_plan* P, int nb, TcBatchA* B) {
    int rc = tc_setup_analysis(P, 2);
    if (rc) return rc;
    const int N = P->N, nh = P->nh;
    TcBatchA T;
    T.nb = nb;
    T.nkt = (nh + TC_TILE_K - 1) / TC_TILE_K;
    const auto per = tile_pieces(N, P->n_ext);
    const auto& cm = tc_chunk_max(P);
    std::vector<int4> items, slots;
    std::vector<double> cost;
    for (int tt = 0; tt < int(per.size()); ++tt) {
        const int np = int(per[tt].size());
        const int ni = std::max(1, 32 / std::max(np, 1));
        for (int j0 = 0; j0 < np; j0 += 32)   // a tile with more than 32 pieces: one instance, 32 pieces per item
            for (int i0 = 0; i0 < nb; i0 += (np > 32 ? 1 : ni)) {
                const int jn = std::min(32, np - j0);
                const int in = np > 32 ? 1 : std::min(ni, nb - i0);
                const int first = int(slots.size());
                for (int j = j0; j < j0 + jn; ++j)
                    for (int k = i0; k < i0 + in; ++k) {
                        const int4 pc = per[tt][j];
                        slots.push_back(make_int4(pc.x, pc.y, k, pc.z | (pc.w << 16)));
                    }
                const int ns = int(slots.size()) - first;
                const int kt0 = ana_first_chunk(cm, T.nkt, tt, per[tt].data() + j0, jn);
                items.push_back(make_int4(tt, first, ns, ((8 * ns + 15) / 16) * 16 | (kt0 << 16)));
                cost.push_back((T.nkt - kt0) * (1.0 + ns / 32.0) + 0.2 * ns);
            }
    }
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    const int G = std::min<int>(P->n_cta, int(items.size()));
    std::vector<std::vector<int4>> bins(G);
    std::vector<double> load(G, 0.0);
    for (int idx : order) {
        const int bb = int(std::min_element(load.begin(), load.end()) - load.begin());
        bins[bb].push_back(items[idx]);
        load[bb] += cost[idx];
    }
    std::vector<int4> flat;
    std::vector<int> offs(1, 0);
    for (auto& bi : bins) {
        flat.insert(flat.end(), bi.begin(), bi.end());
        offs.push_back(int(flat.size()));
    }
    const size_t sbytes = size_t(nb) * 2 * (N + 1) * T.nkt * 1024;
    if (cudaMalloc(reinterpret_cast<void**>(&T.items), flat.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.off), offs.size() * sizeof(int)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.slots), slots.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.stiles), sbytes) != cudaSuccess) {
        tc_batch_ana_free(&T);
        return SPHNSE_E_NOMEM;
    }
    cudaMemcpy(T.items, flat.data(), flat.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(T.off, offs.data(), offs.size() * sizeof(int), cudaMemcpyHostToDevice);
    cudaMemcpy(T.slots, slots.data(), slots.size() * sizeof(int4), cudaMemcpyHostToDevice);
    T.ncta = G;
    *B = T;
    return check_cuda(cudaGetLastError());
}

void tc_batch_ana_free(TcBatchA* B) {
    for (void* q : {static_cast<void*>(B->items), static_cast<void*>(B->off), static_cast<void*>(B->slots),
                    static_cast<void*>(B->stiles)})
        if (q) cudaFree(q);
    *B = TcBatchA();
}

int launch_analysis_tc_batch(sphnse_plan* P, const TcBatchA& B, const float* gana, size_t sa_floats, float* hana,
                             size_t sh_floats) {
    const size_t sm = 1024 + size_t(TC_ANAB_NS) * (2 * size_t(TC_ATILE) + TC_ANAB_BBYTES) + 512;
    if (sm > 227 * 1024) return SPHNSE_E_UNSUPPORTED;
    stage_begin(P, SPHNSE_STAGE_ANALYSIS);
    cudaError_t e = launch_pdl(k_ana_prep, dim3(((P->N + 1) * B.nkt * 16 + 127) / 128, B.nb), dim3(128), 0, P->stream, gana,
                               sa_floats, B.stiles, P->N, P->nh, P->nlat, B.nkt);
    if (e == cudaSuccess) {
        allow_dynamic_smem(reinterpret_cast<const void*>(k_ana_tc_b), sm);
        TcAnaBArgs a{reinterpret_cast<const CUtensorMap*>(P->tc.map_hi),
                     reinterpret_cast<const CUtensorMap*>(P->tc.map_lo), B.items, B.off, B.slots, B.stiles, hana,
                     sh_floats, P->d_status, P->N, B.nkt, P->n_ext};
        e = launch_pdl(k_ana_tc_b, dim3(B.ncta), dim3(192), sm, P->stream, a);
    }
    stage_end(P, SPHNSE_STAGE_ANALYSIS);
    return check_cuda(e);
}

void tc_free(sphnse_plan* P) {
    auto& T = P->tc;
    void* ptrs[] = {T.map_hi, T.map_lo, T.ana_items, T.ana_off, T.ana_pieces, T.anf_items, T.anf_off, T.anf_pieces,
                    T.anf_og, T.anf_map_hi, T.anf_map_lo, T.smap_hi, T.smap_lo, T.tsyn_hi,
                    T.tsyn_lo, T.tile_off, T.tile_info, T.smap_hi_c2, T.smap_lo_c2, T.smap_hi_c4,
                    T.smap_lo_c4};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    tc_batch_free(&T.single);
    T = TcState();
}

}  // namespace sph
