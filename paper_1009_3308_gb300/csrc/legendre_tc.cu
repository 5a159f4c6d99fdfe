// Tensor-core (tcgen05) Legendre analysis with BF16 hi + lo split operands
// and FP32 accumulation in tensor memory.
//
// The per-order analysis of the RHS (Sec. 4.2; the projection of Eq.
// (disc_vec_orth_proj) after the longitude transform) is, per order m and
// parity of K - m, the dense contraction
//     H[K][c] = sum_p Pt_K^m(x_p) S[p][c],   p over the northern nodes,
// with S the hemispheric sum / difference of the weighted Fourier profiles.
// A = table rows (M = degrees, K = latitudes, K-major), B = S (N = columns).
// Split precision: A = A_hi + A_lo, B = B_hi + B_lo (BF16 each), and
//     D = A_hi [B_hi | B_lo] + A_lo [B_hi | 0]      (two MMAs per K step)
// so that H = D[:, 0:c] + D[:, c:2c] = A_hi B_hi + A_hi B_lo + A_lo B_hi.
//
// Tiles: 128 rows x 64 latitudes (one 128-byte swizzle atom column), loaded
// by TMA from one tensor map per (m, parity) block; rows past the block come
// back zero-filled from TMA and are not read from HBM.  B is written by the
// CTA into the same swizzled K-major layout.  Warp roles per CTA: warp 0 TMA
// producer, warp 1 MMA issuer (and TMEM owner), warps 2-5 B builders and
// epilogue (tcgen05.ld of the 128 x 16 FP32 accumulator).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "internal.h"
#include "tc.cuh"

namespace sph {

constexpr int TC_NS = 4;          // A pipeline stages
constexpr int TC_TILE_M = 128;    // rows per MMA tile
constexpr int TC_TILE_K = 64;     // K per smem tile (128 bytes of bf16)
constexpr int TC_N = 16;          // accumulator columns (B rows)
constexpr int TC_ATILE = TC_TILE_M * TC_TILE_K * 2;   // 16 KB
constexpr int TC_BTILE = TC_N * TC_TILE_K * 2;        // 2 KB

struct TcAnaArgs {
    const CUtensorMap* map_hi;   // per (m, parity) block, global memory
    const CUtensorMap* map_lo;
    const int4* items;           // (block, m, parity, row tile)
    const int* item_off;         // per CTA
    const float* gana;           // [NF][N+1][nlat] complex float (m-major)
    float* hana;                 // [n_ext][2 NF]
    unsigned* status;
    int N, nh, nlat, nkt;
};

template <int NF>
__global__ void __launch_bounds__(192, 1) k_ana_tc(TcAnaArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    // 1024-byte aligned base for the swizzled tiles
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~uintptr_t(1023));
    unsigned char* A_hi = smem;                                   // TC_NS x 16 KB
    unsigned char* A_lo = A_hi + TC_NS * TC_ATILE;                // TC_NS x 16 KB
    unsigned char* B1 = A_lo + TC_NS * TC_ATILE;                  // 2 bufs x nkt x 2 KB
    unsigned char* B2 = B1 + 2 * a.nkt * TC_BTILE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(B2 + 2 * a.nkt * TC_BTILE);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + TC_NS;
    uint64_t* b_full = bars + 2 * TC_NS;
    uint64_t* b_empty = b_full + 2;
    uint64_t* acc_full = b_full + 4;
    uint64_t* acc_empty = b_full + 6;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_full + 8);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_NS; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&b_full[b], 128);
            mbar_init(&b_empty[b], 1);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        *abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, 32);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int ib = a.item_off[blockIdx.x], nI = a.item_off[blockIdx.x + 1] - ib;
    const int N = a.N, nh = a.nh, nlat = a.nlat, nkt = a.nkt;

    if (warp == 0) {
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int4 itm = a.items[ib + i];
                for (int kt = 0; kt < nkt; ++kt, ++it) {
                    const int s = it % TC_NS;
                    if (it >= TC_NS && !mbar_wait(&a_empty[s], ((it / TC_NS) - 1) & 1, abort, a.status)) continue;
                    if (*abort) continue;
                    mbar_arrive_expect_tx(&a_full[s], 2 * TC_ATILE);
                    tma_load_2d(A_hi + s * TC_ATILE, &a.map_hi[itm.x], kt * TC_TILE_K, itm.w * TC_TILE_M, &a_full[s], pol);
                    tma_load_2d(A_lo + s * TC_ATILE, &a.map_lo[itm.x], kt * TC_TILE_K, itm.w * TC_TILE_M, &a_full[s], pol);
                }
            }
            for (int k = it - TC_NS; k < it; ++k)
                if (k >= 0) mbar_wait(&a_full[k % TC_NS], (k / TC_NS) & 1, abort, a.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(TC_TILE_M, TC_N);
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int buf = i & 1, use = i >> 1;
                bool ok = mbar_wait(&b_full[buf], use & 1, abort, a.status);
                if (i >= 2) ok = mbar_wait(&acc_empty[buf], (use - 1) & 1, abort, a.status) && ok;
                tc_fence_after();
                const uint32_t d = tmem + uint32_t(buf * TC_N);
                for (int kt = 0; kt < nkt; ++kt, ++it) {
                    const int s = it % TC_NS;
                    const bool okA = mbar_wait(&a_full[s], (it / TC_NS) & 1, abort, a.status);
                    tc_fence_after();
                    if (ok && okA && !*abort) {
#pragma unroll
                        for (int kk = 0; kk < TC_TILE_K / 16; ++kk) {
                            const uint64_t ah = sdesc_sw128(A_hi + s * TC_ATILE + kk * 32);
                            const uint64_t al = sdesc_sw128(A_lo + s * TC_ATILE + kk * 32);
                            const uint64_t b1 = sdesc_sw128(B1 + (buf * nkt + kt) * TC_BTILE + kk * 32);
                            const uint64_t b2 = sdesc_sw128(B2 + (buf * nkt + kt) * TC_BTILE + kk * 32);
                            mma_bf16(d, ah, b1, idesc, (kt | kk) != 0);
                            mma_bf16(d, al, b2, idesc, 1);
                        }
                    }
                    mma_commit(&a_empty[s]);
                }
                mma_commit(&acc_full[buf]);
                mma_commit(&b_empty[buf]);
            }
            if (nI > 0) mbar_wait(&acc_full[(nI - 1) & 1], ((nI - 1) >> 1) & 1, abort, a.status);
        }
    } else {
        // helpers: build B for item i, then drain the accumulator of item i-1
        const int ht = threadIdx.x - 64;
        const int quarter = warp & 3;
        const float* gana = a.gana;
        auto build_B = [&](int i) {
            const int4 itm = a.items[ib + i];
            const int m = itm.y, par = itm.z, buf = i & 1;
            const size_t ld = size_t(N + 1);
            for (int p = ht; p < nkt * TC_TILE_K; p += 128) {
                float v[2 * NF];
#pragma unroll
                for (int f = 0; f < NF; ++f) {
                    float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
                    if (p < nh) {
                        const float* ga = gana + ((size_t(f) * ld + m) * nlat + p) * 2;
                        ar = ga[0];
                        ai = ga[1];
                        const int pr = nlat - 1 - p;
                        if (pr != p) {
                            const float* gb = gana + ((size_t(f) * ld + m) * nlat + pr) * 2;
                            br = gb[0];
                            bi = gb[1];
                        }
                    }
                    v[2 * f] = par ? ar - br : ar + br;
                    v[2 * f + 1] = par ? ai - bi : ai + bi;
                }
                const int kt = p / TC_TILE_K, kl = p % TC_TILE_K;
                unsigned char* t1 = B1 + (buf * nkt + kt) * TC_BTILE;
                unsigned char* t2 = B2 + (buf * nkt + kt) * TC_BTILE;
#pragma unroll
                for (int n = 0; n < TC_N; ++n) {
                    __nv_bfloat16 x1 = __float2bfloat16_rn(0.f), x2 = x1;
                    if (n < 2 * NF) {
                        x1 = __float2bfloat16_rn(v[n]);
                        x2 = x1;
                    } else if (n < 4 * NF) {
                        const float hv = v[n - 2 * NF];
                        x1 = __float2bfloat16_rn(hv - __bfloat162float(__float2bfloat16_rn(hv)));
                    }
                    *reinterpret_cast<__nv_bfloat16*>(t1 + sw128_offset(n, kl)) = x1;
                    *reinterpret_cast<__nv_bfloat16*>(t2 + sw128_offset(n, kl)) = x2;
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&b_full[buf]);
        };
        auto epilogue = [&](int i) {
            const int4 itm = a.items[ib + i];
            const int m = itm.y, par = itm.z, t = itm.w, buf = i & 1;
            const bool ok = mbar_wait(&acc_full[buf], (i >> 1) & 1, abort, a.status);
            tc_fence_after();
            float v[16];
            tmem_ld16(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(buf * TC_N), v);
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);
            const int ne = ext_even(N, m), no = ext_odd(N, m);
            const int nrows = par ? no : ne;
            const int r = t * TC_TILE_M + quarter * 32 + lane;
            if (ok && r < nrows && !*abort) {
                const int row = ext_off(N, m) + (par ? ne : 0) + r;
#pragma unroll
                for (int f = 0; f < 2 * NF; ++f) a.hana[size_t(row) * 2 * NF + f] = v[f] + v[2 * NF + f];
            }
        };
        for (int i = 0; i < nI; ++i) {
            if (i >= 2) mbar_wait(&b_empty[i & 1], ((i >> 1) - 1) & 1, abort, a.status);
            build_B(i);
            if (i >= 1) epilogue(i - 1);
        }
        if (nI > 0) epilogue(nI - 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 32);
    }
}

// ---------------------------------------------------------------------------
// synthesis
//
// Per order m and parity: g[p][c] = sum_j Pt_{K_j}^m(x_p) b[j][c], the dense
// contraction with A = the transposed table block [nh][pad8(n_par)] (M =
// latitudes, K = degrees, K-major; TMA zero-fills degrees past the block),
// B = the coefficient sets of the three fields (N = 16: hi/lo columns as in
// the analysis).  Both parities of an order go to separate accumulators so
// that the epilogue forms north = E + O, south = E - O directly.

struct TcSynArgs {
    const CUtensorMap* map_hi;   // per (m, parity) block of the transposed tables
    const CUtensorMap* map_lo;
    const int* items;            // orders m per CTA (LPT)
    const int* item_off;
    const float* bsyn;           // [n_ext][6]
    float* gsyn;                 // [3][N+1][nlat] complex (m-major)
    const double* sinth;
    unsigned* status;
    int N, nh, nlat, nmt, maxkt;
};

constexpr int TC_SYN_COLS = 256;  // TMEM columns: 2 buffers x 2 parities x nmt (<= 4) x 16

__global__ void __launch_bounds__(192, 1) k_syn_tc(TcSynArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                                           ~uintptr_t(1023));
    const int maxkt = a.maxkt, nmt = a.nmt;
    unsigned char* A_hi = smem;
    unsigned char* A_lo = A_hi + TC_NS * TC_ATILE;
    unsigned char* B1 = A_lo + TC_NS * TC_ATILE;                 // [buf][par][kt] x 2 KB
    unsigned char* B2 = B1 + 2 * 2 * maxkt * TC_BTILE;
    uint64_t* bars = reinterpret_cast<uint64_t*>(B2 + 2 * 2 * maxkt * TC_BTILE);
    uint64_t* a_full = bars;
    uint64_t* a_empty = bars + TC_NS;
    uint64_t* b_full = bars + 2 * TC_NS;
    uint64_t* b_empty = b_full + 2;
    uint64_t* acc_full = b_full + 4;
    uint64_t* acc_empty = b_full + 6;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(b_full + 8);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_NS; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&b_full[b], 128);
            mbar_init(&b_empty[b], 1);
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 128);
        }
        *abort = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, TC_SYN_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int ib = a.item_off[blockIdx.x], nI = a.item_off[blockIdx.x + 1] - ib;
    const int N = a.N, nh = a.nh, nlat = a.nlat;
    auto nkt_of = [&](int m, int par) {
        const int n = par ? ext_odd(N, m) : ext_even(N, m);
        return (((n + 7) / 8) * 8 + TC_TILE_K - 1) / TC_TILE_K;
    };

    if (warp == 0) {
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int m = a.items[ib + i];
                for (int par = 0; par < 2; ++par) {
                    const int b = 2 * m + par, nkt = nkt_of(m, par);
                    for (int kt = 0; kt < nkt; ++kt)
                        for (int mt = 0; mt < nmt; ++mt, ++it) {
                            const int s = it % TC_NS;
                            if (it >= TC_NS && !mbar_wait(&a_empty[s], ((it / TC_NS) - 1) & 1, abort, a.status))
                                continue;
                            if (*abort) continue;
                            mbar_arrive_expect_tx(&a_full[s], 2 * TC_ATILE);
                            tma_load_2d(A_hi + s * TC_ATILE, &a.map_hi[b], kt * TC_TILE_K, mt * TC_TILE_M, &a_full[s], pol);
                            tma_load_2d(A_lo + s * TC_ATILE, &a.map_lo[b], kt * TC_TILE_K, mt * TC_TILE_M, &a_full[s], pol);
                        }
                }
            }
            for (int k = it - TC_NS; k < it; ++k)
                if (k >= 0) mbar_wait(&a_full[k % TC_NS], (k / TC_NS) & 1, abort, a.status);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(TC_TILE_M, TC_N);
            int it = 0;
            for (int i = 0; i < nI; ++i) {
                const int m = a.items[ib + i];
                const int buf = i & 1, use = i >> 1;
                bool ok = mbar_wait(&b_full[buf], use & 1, abort, a.status);
                if (i >= 2) ok = mbar_wait(&acc_empty[buf], (use - 1) & 1, abort, a.status) && ok;
                tc_fence_after();
                for (int par = 0; par < 2; ++par) {
                    const int nkt = nkt_of(m, par);
                    for (int kt = 0; kt < nkt; ++kt)
                        for (int mt = 0; mt < nmt; ++mt, ++it) {
                            const int s = it % TC_NS;
                            const bool okA = mbar_wait(&a_full[s], (it / TC_NS) & 1, abort, a.status);
                            tc_fence_after();
                            const uint32_t d = tmem + uint32_t(((buf * 2 + par) * nmt + mt) * TC_N);
                            if (ok && okA && !*abort) {
                                const unsigned char* bt1 = B1 + ((buf * 2 + par) * maxkt + kt) * TC_BTILE;
                                const unsigned char* bt2 = B2 + ((buf * 2 + par) * maxkt + kt) * TC_BTILE;
#pragma unroll
                                for (int kk = 0; kk < TC_TILE_K / 16; ++kk) {
                                    mma_bf16(d, sdesc_sw128(A_hi + s * TC_ATILE + kk * 32), sdesc_sw128(bt1 + kk * 32),
                                             idesc, (kt | kk) != 0);
                                    mma_bf16(d, sdesc_sw128(A_lo + s * TC_ATILE + kk * 32), sdesc_sw128(bt2 + kk * 32),
                                             idesc, 1);
                                }
                            }
                            mma_commit(&a_empty[s]);
                        }
                }
                mma_commit(&acc_full[buf]);
                mma_commit(&b_empty[buf]);
            }
            if (nI > 0) mbar_wait(&acc_full[(nI - 1) & 1], ((nI - 1) >> 1) & 1, abort, a.status);
        }
    } else {
        const int ht = threadIdx.x - 64;
        const int quarter = warp & 3;
        auto build_B = [&](int i) {
            const int m = a.items[ib + i], buf = i & 1;
            const int ne = ext_even(N, m), e0 = ext_off(N, m);
            for (int par = 0; par < 2; ++par) {
                const int n = par ? ext_odd(N, m) : ne;
                const int nk = nkt_of(m, par) * TC_TILE_K;
                for (int j = ht; j < nk; j += 128) {
                    float v[6];
                    if (j < n) {
                        const float* src = a.bsyn + size_t(e0 + (par ? ne : 0) + j) * 6;
#pragma unroll
                        for (int c = 0; c < 6; ++c) v[c] = src[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 6; ++c) v[c] = 0.f;
                    }
                    const int kt = j / TC_TILE_K, kl = j % TC_TILE_K;
                    unsigned char* t1 = B1 + ((buf * 2 + par) * maxkt + kt) * TC_BTILE;
                    unsigned char* t2 = B2 + ((buf * 2 + par) * maxkt + kt) * TC_BTILE;
#pragma unroll
                    for (int c = 0; c < TC_N; ++c) {
                        __nv_bfloat16 x1 = __float2bfloat16_rn(0.f), x2 = x1;
                        if (c < 6) {
                            x1 = __float2bfloat16_rn(v[c]);
                            x2 = x1;
                        } else if (c < 12) {
                            x1 = __float2bfloat16_rn(v[c - 6] - __bfloat162float(__float2bfloat16_rn(v[c - 6])));
                        }
                        *reinterpret_cast<__nv_bfloat16*>(t1 + sw128_offset(c, kl)) = x1;
                        *reinterpret_cast<__nv_bfloat16*>(t2 + sw128_offset(c, kl)) = x2;
                    }
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&b_full[buf]);
        };
        auto epilogue = [&](int i) {
            const int m = a.items[ib + i], buf = i & 1;
            const bool ok = mbar_wait(&acc_full[buf], (i >> 1) & 1, abort, a.status);
            tc_fence_after();
            const float mm = float(m);
            const size_t ld = size_t(N + 1);
            for (int mt = 0; mt < nmt; ++mt) {
                float E[16], O[16];
                const uint32_t lanes = uint32_t(quarter * 32) << 16;
                tmem_ld16(tmem + lanes + uint32_t(((buf * 2 + 0) * nmt + mt) * TC_N), E);
                tmem_ld16(tmem + lanes + uint32_t(((buf * 2 + 1) * nmt + mt) * TC_N), O);
                const int p = mt * TC_TILE_M + quarter * 32 + lane;
                if (!ok || p >= nh || *abort) continue;
                const float inv_s = float(1.0 / a.sinth[p]);
#pragma unroll
                for (int hemi = 0; hemi < 2; ++hemi) {
                    const int row = hemi == 0 ? p : nlat - 1 - p;
                    if (hemi == 1 && row == p) break;
                    const float sg = hemi == 0 ? 1.f : -1.f;
#pragma unroll
                    for (int f = 0; f < 3; ++f) {
                        const float gr = (E[2 * f] + E[6 + 2 * f]) + sg * (O[2 * f] + O[6 + 2 * f]);
                        const float gi = (E[2 * f + 1] + E[7 + 2 * f]) + sg * (O[2 * f + 1] + O[7 + 2 * f]);
                        float o0, o1;
                        if (f == 0) { o0 = gr; o1 = gi; }
                        else if (f == 1) { o0 = -mm * gi * inv_s; o1 = mm * gr * inv_s; }
                        else { o0 = -gr * inv_s; o1 = -gi * inv_s; }
                        float* d = a.gsyn + ((size_t(f) * ld + m) * nlat + row) * 2;
                        d[0] = o0;
                        d[1] = o1;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&acc_empty[buf]);
        };
        for (int i = 0; i < nI; ++i) {
            if (i >= 2) mbar_wait(&b_empty[i & 1], ((i >> 1) - 1) & 1, abort, a.status);
            build_B(i);
            if (i >= 1) epilogue(i - 1);
        }
        if (nI > 0) epilogue(nI - 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TC_SYN_COLS);
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

bool tc_supported(const sphnse_plan* P) { return P->nh % 8 == 0 && P->nh >= 64 && P->nlat % 2 == 0; }

// Tensor maps over every (m, parity) block of the [ext row][nh] bf16 tables,
// and the LPT schedule of (block, row tile) items over one CTA per SM.
int tc_setup_analysis(sphnse_plan* P) {
    if (P->tc.ana_ready) return SPHNSE_OK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return SPHNSE_E_UNSUPPORTED;
    const Tables& t = P->tab[SPHNSE_BF16X3];
    const int N = P->N, nh = P->nh;
    const int nblk = 2 * (N + 1);
    std::vector<CUtensorMap> mh(nblk), ml(nblk);
    std::vector<int4> items;
    std::vector<int> cost;
    for (int m = 0; m <= N; ++m) {
        for (int par = 0; par < 2; ++par) {
            const int ne = ext_even(N, m), no = ext_odd(N, m);
            const int nrows = par ? no : ne;
            const int r0 = ext_off(N, m) + (par ? ne : 0);
            const int b = 2 * m + par;
            const cuuint64_t dims[2] = {cuuint64_t(nh), cuuint64_t(nrows)};
            const cuuint64_t strides[1] = {cuuint64_t(nh) * 2};
            const cuuint32_t box[2] = {TC_TILE_K, TC_TILE_M};
            const cuuint32_t es[2] = {1, 1};
            for (int lo = 0; lo < 2; ++lo) {
                const __nv_bfloat16* base = reinterpret_cast<const __nv_bfloat16*>(lo ? t.syn_lo : t.syn) +
                                            size_t(r0) * nh;
                CUresult r = enc(lo ? &ml[b] : &mh[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(base),
                                 dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
                if (r != CUDA_SUCCESS) return SPHNSE_E_CUDA;
            }
            for (int tt = 0; tt * TC_TILE_M < nrows; ++tt) {
                items.push_back(make_int4(b, m, par, tt));
                cost.push_back(std::min(TC_TILE_M, nrows - tt * TC_TILE_M) + 16);
            }
        }
    }
    // LPT: largest items first onto the least-loaded CTA
    std::vector<int> order(items.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = int(i);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    const int G = std::min<int>(P->n_cta, int(items.size()));
    std::vector<std::vector<int4>> bins(G);
    std::vector<long> load(G, 0);
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
    auto& T = P->tc;
    if (cudaMalloc(&T.map_hi, nblk * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(&T.map_lo, nblk * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.ana_items), flat.size() * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(reinterpret_cast<void**>(&T.ana_off), off.size() * sizeof(int)) != cudaSuccess)
        return SPHNSE_E_NOMEM;
    cudaMemcpy(T.map_hi, mh.data(), nblk * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    cudaMemcpy(T.map_lo, ml.data(), nblk * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    cudaMemcpy(T.ana_items, flat.data(), flat.size() * sizeof(int4), cudaMemcpyHostToDevice);
    cudaMemcpy(T.ana_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice);
    T.ana_cta = G;
    T.ana_ready = true;
    return check_cuda(cudaGetLastError());
}

template <int NF>
static int ana_tc_t(sphnse_plan* P) {
    const int nkt = (P->nh + TC_TILE_K - 1) / TC_TILE_K;
    const size_t sm = 1024 + 2 * size_t(TC_NS) * TC_ATILE + 4 * size_t(nkt) * TC_BTILE + 256;
    if (sm > 227 * 1024) return SPHNSE_E_UNSUPPORTED;
    cudaFuncSetAttribute(k_ana_tc<NF>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    TcAnaArgs a{reinterpret_cast<const CUtensorMap*>(P->tc.map_hi), reinterpret_cast<const CUtensorMap*>(P->tc.map_lo), P->tc.ana_items, P->tc.ana_off,
                reinterpret_cast<const float*>(P->d_gana), reinterpret_cast<float*>(P->d_hana), P->d_status,
                P->N, P->nh, P->nlat, nkt};
    stage_begin(P, SPHNSE_STAGE_ANALYSIS);
    k_ana_tc<NF><<<P->tc.ana_cta, 192, sm, P->stream>>>(a);
    stage_end(P, SPHNSE_STAGE_ANALYSIS);
    return check_cuda(cudaGetLastError());
}

int launch_analysis_tc(sphnse_plan* P, int nfields) {
    int rc = tc_setup_analysis(P);
    if (rc) return rc;
    return nfields == 3 ? ana_tc_t<3>(P) : ana_tc_t<2>(P);
}

// Transposed, padded bf16 hi/lo tables for the synthesis (block (m, parity)
// stored [nh][pad8(n_par)]) and their tensor maps.
int tc_setup_synthesis(sphnse_plan* P) {
    if (P->tc.syn_ready) return SPHNSE_OK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return SPHNSE_E_UNSUPPORTED;
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
    std::vector<CUtensorMap> mh(nblk), ml(nblk);
    for (int b = 0; b < nblk; ++b) {
        const int m = b / 2, par = b % 2;
        const int n = par ? ext_odd(N, m) : ext_even(N, m);
        const int np = ((n + 7) / 8) * 8;
        const cuuint64_t dims[2] = {cuuint64_t(np), cuuint64_t(nh)};
        const cuuint64_t strides[1] = {cuuint64_t(np) * 2};
        const cuuint32_t box[2] = {TC_TILE_K, TC_TILE_M};
        const cuuint32_t es[2] = {1, 1};
        for (int l = 0; l < 2; ++l) {
            __nv_bfloat16* base = reinterpret_cast<__nv_bfloat16*>(l ? T.tsyn_lo : T.tsyn_hi) + off[b];
            CUresult r = enc(l ? &ml[b] : &mh[b], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return SPHNSE_E_CUDA;
        }
    }
    if (cudaMalloc(&T.smap_hi, nblk * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(&T.smap_lo, nblk * sizeof(CUtensorMap)) != cudaSuccess)
        return SPHNSE_E_NOMEM;
    cudaMemcpy(T.smap_hi, mh.data(), nblk * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    cudaMemcpy(T.smap_lo, ml.data(), nblk * sizeof(CUtensorMap), cudaMemcpyHostToDevice);
    T.tsyn_bytes = 2 * total * 2;
    T.syn_ready = true;
    return check_cuda(cudaGetLastError());
}

int launch_synthesis_tc(sphnse_plan* P) {
    int rc = tc_setup_synthesis(P);
    if (rc) return rc;
    const int nmt = (P->nh + TC_TILE_M - 1) / TC_TILE_M;
    if (nmt > 4) return SPHNSE_E_UNSUPPORTED;
    const int maxkt = (((ext_even(P->N, 0) + 7) / 8) * 8 + TC_TILE_K - 1) / TC_TILE_K;
    const size_t sm = 1024 + 2 * size_t(TC_NS) * TC_ATILE + 8 * size_t(maxkt) * TC_BTILE + 256;
    if (sm > 227 * 1024) return SPHNSE_E_UNSUPPORTED;
    cudaFuncSetAttribute(k_syn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
    TcSynArgs a{reinterpret_cast<const CUtensorMap*>(P->tc.smap_hi),
                reinterpret_cast<const CUtensorMap*>(P->tc.smap_lo), P->d_items, P->d_item_off,
                reinterpret_cast<const float*>(P->d_bsyn), reinterpret_cast<float*>(P->d_gsyn), P->d_s,
                P->d_status, P->N, P->nh, P->nlat, nmt, maxkt};
    stage_begin(P, SPHNSE_STAGE_SYNTHESIS);
    k_syn_tc<<<P->n_cta, 192, sm, P->stream>>>(a);
    stage_end(P, SPHNSE_STAGE_SYNTHESIS);
    return check_cuda(cudaGetLastError());
}

void tc_free(sphnse_plan* P) {
    auto& T = P->tc;
    void* ptrs[] = {T.map_hi, T.map_lo, T.ana_items, T.ana_off, T.smap_hi, T.smap_lo, T.tsyn_hi, T.tsyn_lo};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    T = TcState();
}

}  // namespace sph
