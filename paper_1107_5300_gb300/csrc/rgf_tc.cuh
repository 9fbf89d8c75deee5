// rgf_tc.cuh -- complex matrix products on the tcgen05 tensor cores at
// double-float accuracy (the dense contractions of the RGF step: the rank-b
// updates of the slice inverse and the corner-strip product of Eq. 5).
//
// Method: exact digit slicing (the Ozaki scheme; K. Ozaki, T. Ogita, S. Oishi,
// S. M. Rump, Numer. Algorithms 59 (2012) 95).  Each row of A (each column of
// B) gets a power-of-two scale 2^e with |entries| < 2^e.  A real double-float
// value x of that row is written as a sum of S signed base-256 digits,
//     x ~ 2^(e-7) sum_i d_i 2^(-8 i),   d_i integer, |d_i| <= 128,
// every digit exact in bfloat16.  The tile of digit i holds d_i 2^(-8 i).
// A product of digit tiles i (of A) and j (of B) carries the weight
// 2^(-8 (i + j)); the tensor core accumulates it in binary32:
//     level l = i + j = 0 .. 3    one TMEM accumulator each.  Every term of a
//                                 level is an integer multiple of 2^(-8 l)
//                                 below 2^14, and a level sums at most
//                                 4 x 256 x 2^14 = 2^24 of them: exact;
//     levels 4 .. S-1             one shared accumulator.  The tensor core's
//                                 binary32 additions drop low-order bits at
//                                 every MMA (measured: sharing it with level 3
//                                 cost 2^-44 of the scale); at 2^-32 of the
//                                 scale these levels lose less than 2^-50;
//     levels >= S                 dropped (below 2^-(8S-1) of the scale).
// The five accumulators are combined in double-float (error-free sums) and
// scaled back by 2^(e_row - 7) 2^(e_col - 7).  With S = 7 digits (55 bits)
// the product is accurate to a few units of 2^-48 of (row max x column max x
// inner dimension), the accuracy of the double-float arithmetic it replaces.
//
// Complex products use the real 2 x 2 block form
//     [Re C | Im C] = A' B',  A'[m][2k] = Re A, A'[m][2k+1] = Im A,
//     B'[2k][n] = Re B, B'[2k+1][n] = -Im B  (Re columns),
//     B'[2k][n'] = Im B, B'[2k+1][n'] = Re B (Im columns),
// so one MMA chain (M = 128, N = 2 x columns, K = 16 per instruction, bf16 x
// bf16 -> f32) gives both parts.  Operands are staged in shared memory by the
// threads that slice them (K-major, no swizzle: 8-row x 16-byte core
// matrices, 128 B apart along K and 256 B apart along M/N); one elected
// thread issues the MMAs and commits them to an mbarrier; the accumulators
// live in TMEM (5 x 96 columns) and are read back with tcgen05.ld.
#pragma once

#include <cuda_bf16.h>

#include "rgf_common.cuh"

namespace rgf {
namespace tc {

constexpr int S = 7;                 // digits per real value
constexpr int TILE = 128 * 16;       // elements of one operand tile (128 rows x 16 k)
constexpr int NACC = 5;              // TMEM accumulators: levels 0..3 exact, 4.. shared
constexpr int MAXC = 48;             // complex output columns per pass
constexpr int ACOLS = 2 * MAXC;      // TMEM columns per accumulator (5 x 96 <= 512)
constexpr int KCH = 8;               // complex inner entries per chunk (16 real-block k)
constexpr int KGRP = 128;            // complex inner entries per exact accumulation group

struct Smem {
    __nv_bfloat16* a;     // [S][TILE]  digit tiles of A'
    __nv_bfloat16* b;     // [S][TILE]  digit tiles of B'
    float* rsc;           // [128] row slicing scale 2^(7-e)
    float* rfac;          // [128] row output factor 2^(e-7)
    float* csc;           // [MAXC] column slicing scale
    float* cfac;          // [MAXC] column output factor
    unsigned* cmax;       // [MAXC] column maxima (binary32 bits)
    unsigned long long* bar;   // MMA completion mbarrier
    uint32_t* tslot;      // TMEM base address (written by tcgen05.alloc)
    int* err;             // sticky: an MMA wait gave up
};

// Per-thread view of the tensor-core area plus the mbarrier phase this
// thread expects next (every thread waits on every commit).
struct State {
    Smem s;
    uint32_t phase;
};

__host__ __device__ constexpr size_t smem_bytes() {
    return (size_t)2 * S * TILE * 2 + 2 * 128 * 4 + 3 * MAXC * 4 + 64;
}

// Carves the tensor-core area from `base` (1024-byte aligned offsets inside).
__device__ inline Smem carve(unsigned char* base) {
    Smem s;
    s.a = reinterpret_cast<__nv_bfloat16*>(base);
    s.b = s.a + S * TILE;
    float* f = reinterpret_cast<float*>(s.b + S * TILE);
    s.rsc = f;
    s.rfac = f + 128;
    s.csc = f + 256;
    s.cfac = s.csc + MAXC;
    s.cmax = reinterpret_cast<unsigned*>(s.cfac + MAXC);
    s.bar = reinterpret_cast<unsigned long long*>(s.cmax + MAXC);
    s.tslot = reinterpret_cast<uint32_t*>(s.bar + 1);
    s.err = reinterpret_cast<int*>(s.tslot + 1);
    return s;
}

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Element offset of (row r, k) inside one 128 x 16 K-major tile.
__device__ __forceinline__ int tile_off(int r, int k) {
    return (r >> 3) * 128 + (k >> 3) * 64 + (r & 7) * 8 + (k & 7);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset 128 (next core matrix along K), stride-dimension byte offset 256
// (next 8-row group), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(const void* p) {
    return (uint64_t)((su32(p) >> 4) & 0x3FFFu) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(256 >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: D f32, A and B bf16, both K-major,
// M = 128, N = n (multiple of 16, <= 256).
__device__ __forceinline__ uint32_t idesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
                 :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void commit(unsigned long long* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(su32(bar)) : "memory");
}

__device__ __forceinline__ bool try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok) : "r"(su32(bar)), "r"(parity) : "memory");
    return ok != 0;
}

// 32 lanes x 8 consecutive columns of TMEM (this warp's lane quarter).
__device__ __forceinline__ void ld8(uint32_t addr, float* v) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(addr));
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Allocates all 512 TMEM columns (warp 0) and initialises the mbarrier.  Must
// be called by every thread of the block (it ends with a barrier); the block
// must be the only one on its SM that uses TMEM.  Returns the initial phase.
__device__ inline uint32_t setup(const Smem& s) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     :: "r"(su32(s.tslot)) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(s.bar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *s.err = 0;
    }
    fence_before();
    __syncthreads();
    fence_after();
    return 0u;
}

// Releases TMEM.  Every thread; no MMA may be in flight.
__device__ inline void teardown(const Smem& s) {
    fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(*s.tslot) : "memory");
}

// Waits (every thread) for the MMAs committed last; gives up after about a
// second of device clock and sets the sticky error flag, after which later
// waits return at once.
__device__ inline void wait_mma(const Smem& s, uint32_t& phase) {
    if (!*(volatile int*)s.err) {
        bool done = try_wait(s.bar, phase);
        if (!done) {
            const long long t0 = clock64();
            while (!done) {
                done = try_wait(s.bar, phase);
                if (!done && clock64() - t0 > 2000000000ll) break;
            }
            if (!done) *(volatile int*)s.err = 1;
        }
    }
    phase ^= 1u;
    fence_after();
}

// The S signed base-256 digits of the double-float value (h, l) times the
// slicing scale sc (|h sc| < 128 + 1).  Each step takes the nearest integer of
// the remainder, subtracts it exactly and renormalises the remainder with an
// error-free sum before the next factor 256.
__device__ __forceinline__ void digits(float h, float l, float sc, float* d) {
    float x = __fmul_rn(h, sc), y = __fmul_rn(l, sc);
#pragma unroll
    for (int i = 0; i < S; ++i) {
        const float di = rintf(__fadd_rn(x, y));
        d[i] = di;
        float s2, e2;
        two_sum(__fsub_rn(x, di), y, s2, e2);
        x = __fmul_rn(s2, 256.0f);
        y = __fmul_rn(e2, 256.0f);
    }
}

// Weight of digit i inside its tile.
__device__ __forceinline__ float dweight(int i) { return __int_as_float((127 - 8 * i) << 23); }

// Max with NaN propagation (non-negative arguments).
__device__ __forceinline__ float nmax(float a, float b) { return (isnan(b) || b > a) ? b : a; }

// Slicing scale and output factor for a row / column maximum mx.
__device__ __forceinline__ void scales(float mx, float& sc, float& fac) {
    if (!(mx <= 3.0e38f)) {          // NaN or Inf: poison the outputs of this row / column
        sc = 1.0f;
        fac = __int_as_float(0x7fc00000);
        return;
    }
    int e = 0;
    frexpf(mx, &e);                  // mx < 2^e (e = 0 for mx = 0)
    if (e < -100) {                  // below any value this path meets: treat as zero
        sc = 0.0f;
        fac = 0.0f;
        return;
    }
    sc = ldexpf(1.0f, 7 - e);
    fac = ldexpf(1.0f, e - 7);
}

// The accumulators of one (row, column) -> double-float value, scaled.  The
// exact levels are summed error-free (their rounding errors are multiples of
// 2^-24 small enough to add exactly into t); the shared one is added last.
__device__ __forceinline__ df32 combine(float a0, float a1, float a2, float a3, float a4, float f) {
    float s, t, s2, e2, s3, e3;
    two_sum(a0, a1, s, t);
    two_sum(s, a2, s2, e2);
    two_sum(s2, a3, s3, e3);
    t = __fadd_rn(__fadd_rn(__fadd_rn(t, e2), e3), a4);
    df32 r;
    fast_two_sum(s3, t, r.hi, r.lo);
    r.hi = __fmul_rn(r.hi, f);
    r.lo = __fmul_rn(r.lo, f);
    return r;
}

// C op= A B, A: M x Kc (M <= 128), B: Kc x N, complex double-float, through the
// accessor object `op`:
//   zf  op.a(m, k), op.b(k, n)                      operand entries
//   void op.out(m, n, part, df32 v, bool first)     v = Re (part 0) or Im (part 1)
//                                                   of (A B)[m][n] over one group
//                                                   of up to 128 inner entries;
//                                                   first = the first group.
// Called by every thread of the block (NT = 512); ends with a barrier.
template <class Op>
__device__ __noinline__ void zgemm(Op& op, int M, int N, int Kc, const Smem& s, uint32_t& phase) {
    static_assert(NT == 512, "zgemm assumes 512 threads");
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tmem = *s.tslot;
    for (int g0 = 0; g0 < Kc; g0 += KGRP) {
        const int kg = min(KGRP, Kc - g0);
        // row scales over this group
        for (int m = warp; m < 128; m += NWARP) {
            float mx = 0.0f;
            if (m < M)
                for (int k = lane; k < kg; k += 32) {
                    const zf v = op.a(m, g0 + k);
                    mx = nmax(mx, nmax(fabsf(v.re.hi), fabsf(v.im.hi)));
                }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mx = nmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) scales(mx, s.rsc[m], s.rfac[m]);
        }
        for (int n0 = 0; n0 < N; n0 += MAXC) {
            const int nc = min(MAXC, N - n0);
            const int ncp = (nc + 7) & ~7;
            const int NR = 2 * ncp;               // real output columns [Re ncp | Im ncp]
            if (tid < MAXC) s.cmax[tid] = 0u;
            __syncthreads();
            if (tid < (NT / MAXC) * MAXC) {
                const int c = tid % MAXC, ks = tid / MAXC;
                float mx = 0.0f;
                if (c < nc)
                    for (int k = ks; k < kg; k += NT / MAXC) {
                        const zf v = op.b(g0 + k, n0 + c);
                        mx = nmax(mx, nmax(fabsf(v.re.hi), fabsf(v.im.hi)));
                    }
                if (c < nc) atomicMax(&s.cmax[c], __float_as_uint(mx));
            }
            __syncthreads();
            if (tid < MAXC) scales(__uint_as_float(s.cmax[tid]), s.csc[tid], s.cfac[tid]);
            __syncthreads();
            uint32_t init = 0u;
            for (int k0 = 0; k0 < kg; k0 += KCH) {
                // A': 128 rows x 8 complex entries, two per thread
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int e = tid + h * NT, m = e >> 3, k = e & 7;
                    float dr[S], di[S];
                    if (m < M && k0 + k < kg) {
                        const zf v = op.a(m, g0 + k0 + k);
                        const float sc = s.rsc[m];
                        digits(v.re.hi, v.re.lo, sc, dr);
                        digits(v.im.hi, v.im.lo, sc, di);
                    } else {
#pragma unroll
                        for (int i = 0; i < S; ++i) { dr[i] = 0.0f; di[i] = 0.0f; }
                    }
                    const int o = tile_off(m, 2 * k);
#pragma unroll
                    for (int i = 0; i < S; ++i) {
                        const float w = dweight(i);
                        *reinterpret_cast<__nv_bfloat162*>(s.a + i * TILE + o) =
                            __floats2bfloat162_rn(dr[i] * w, di[i] * w);
                    }
                }
                // B': 8 complex entries x ncp columns, one per thread
                {
                    const int k = tid >> 6, c = tid & 63;
                    if (c < ncp) {
                        float dr[S], di[S];
                        if (c < nc && k0 + k < kg) {
                            const zf v = op.b(g0 + k0 + k, n0 + c);
                            const float sc = s.csc[c];
                            digits(v.re.hi, v.re.lo, sc, dr);
                            digits(v.im.hi, v.im.lo, sc, di);
                        } else {
#pragma unroll
                            for (int i = 0; i < S; ++i) { dr[i] = 0.0f; di[i] = 0.0f; }
                        }
                        const int ore = tile_off(c, 2 * k), oim = tile_off(ncp + c, 2 * k);
#pragma unroll
                        for (int i = 0; i < S; ++i) {
                            const float w = dweight(i);
                            *reinterpret_cast<__nv_bfloat162*>(s.b + i * TILE + ore) =
                                __floats2bfloat162_rn(dr[i] * w, -di[i] * w);
                            *reinterpret_cast<__nv_bfloat162*>(s.b + i * TILE + oim) =
                                __floats2bfloat162_rn(di[i] * w, dr[i] * w);
                        }
                    }
                }
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    fence_after();
                    const uint32_t id = idesc(NR);
#pragma unroll
                    for (int l = 0; l < S; ++l)
#pragma unroll
                        for (int i = 0; i <= l; ++i) {
                            const int j = l - i, acc = l < NACC - 1 ? l : NACC - 1;
                            mma(tmem + (uint32_t)(ACOLS * acc), sdesc(s.a + i * TILE), sdesc(s.b + j * TILE), id,
                                (init >> acc) & 1u);
                            init |= 1u << acc;
                        }
                    commit(s.bar);
                }
                wait_mma(s, phase);     // tiles may be rewritten; accumulators final
                init = (1u << NACC) - 1u;
            }
            // drain: warp w reads lanes 32 (w & 3) .. +31 (rows) and every
            // fourth 8-column block starting at block w >> 2
            {
                const int q = warp & 3, m = 32 * q + lane;
                const float rf = s.rfac[m];
                for (int cb = warp >> 2; cb < NR / 8; cb += 4) {
                    float a0[8], a1[8], a2[8], a3[8], a4[8];
                    const uint32_t ad = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(8 * cb);
                    ld8(ad, a0);
                    ld8(ad + ACOLS, a1);
                    ld8(ad + 2 * ACOLS, a2);
                    ld8(ad + 3 * ACOLS, a3);
                    ld8(ad + 4 * ACOLS, a4);
                    ld_wait();
                    if (m < M) {
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const int col = 8 * cb + j;
                            const int part = col >= ncp ? 1 : 0;
                            const int c = col - part * ncp;
                            if (c < nc) {
                                const df32 v = combine(a0[j], a1[j], a2[j], a3[j], a4[j], rf * s.cfac[c]);
                                op.out(m, n0 + c, part, v, g0 == 0);
                            }
                        }
                    }
                }
            }
            fence_before();
            __syncthreads();            // accumulators read; next pass may overwrite
        }
    }
}

}  // namespace tc
}  // namespace rgf
