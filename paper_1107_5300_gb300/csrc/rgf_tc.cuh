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
//     level l = i + j = 0 .. 4    one TMEM accumulator each.  Every term of a
//                                 level is an integer multiple of 2^(-8 l)
//                                 below 2^14, and a level sums at most
//                                 5 x 192 of them (groups of up to 96 complex
//                                 inner entries): below 2^24, exact;
//     levels 5 .. S-1             one shared accumulator.  The tensor core's
//                                 binary32 additions drop low-order bits at
//                                 every MMA (measured: sharing it with level 3
//                                 cost 2^-44 of the scale, with level 4 about
//                                 2^-48 over the 288 MMAs of a 123-deep
//                                 product); at 2^-40 of the scale these
//                                 levels lose less than 2^-55;
//     levels >= S                 dropped (below 2^-(8S-1) of the scale).
// The six accumulators are summed in double-float and scaled back by
// 2^(e_row - 7) 2^(e_col - 7).  With S = 7 digits (55 bits)
// the product is accurate to a few units of 2^-48 of (row max x column max x
// inner dimension), the accuracy of the double-float arithmetic it replaces.
//
// Complex products use the real 2 x 2 block form C' = A' B' with
//     A'[m][2k] = Re A[m][k],  A'[m][2k+1] = Im A[m][k],
//     B'[2k][2n] = Re B[k][n], B'[2k+1][2n] = -Im B[k][n]      (C'[m][2n] = Re C),
//     B'[2k][2n+1] = Im B[k][n], B'[2k+1][2n+1] = Re B[k][n]   (C'[m][2n+1] = Im C),
// so one MMA chain (M = 128, N = 2 x columns, K = 16 per instruction, bf16 x
// bf16 -> f32) gives both parts, side by side in TMEM.  Operands are staged in shared memory by the
// threads that slice them (K-major, no swizzle: 8-row x 16-byte core
// matrices, 128 B apart along K and 256 B apart along M/N); one elected
// thread issues the MMAs and commits them to an mbarrier; the accumulators
// live in TMEM (6 x 80 columns) and are read back with tcgen05.ld.
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "rgf_common.cuh"

namespace rgf {
namespace tc {

constexpr int S = 7;                 // digits per real value
constexpr int TILE = 128 * 16;       // elements of one operand tile (128 rows x 16 k)
constexpr int NACC = 6;              // TMEM accumulators: levels 0..4 exact, 5.. shared
constexpr int MAXC = 40;             // complex output columns per pass
constexpr int ACOLS = 2 * MAXC;      // TMEM columns per accumulator (6 x 80 <= 512)
constexpr int KCH = 8;               // complex inner entries per chunk (16 real-block k)
constexpr int KGRP = 96;             // complex inner entries per exact accumulation group
constexpr int NCA = 2;               // chunks of A' whose digit tiles stay resident across passes

// Byte offsets inside the tensor-core area of shared memory.
constexpr int OFF_A = 0;                          // [NCA][S][TILE] bf16 digit tiles of A'
constexpr int OFF_B = OFF_A + NCA * S * TILE * 2; // [S][TILE] bf16 digit tiles of B'
constexpr int OFF_RSC = OFF_B + S * TILE * 2;     // [128] row slicing scales 2^(7-e)
constexpr int OFF_RFAC = OFF_RSC + 128 * 4;       // [128] row output factors 2^(e-7)
constexpr int OFF_CSC = OFF_RFAC + 128 * 4;       // [MAXC] column slicing scales
constexpr int OFF_CFAC = OFF_CSC + MAXC * 4;      // [MAXC] column output factors
constexpr int OFF_CMAX = OFF_CFAC + MAXC * 4;     // [MAXC] column maxima (binary32 bits)
constexpr int OFF_BAR = OFF_CMAX + MAXC * 4;      // MMA completion mbarrier (8 bytes)
constexpr int OFF_BAR2 = OFF_BAR + 8;             // drain mbarrier after a timeout (8 bytes)
constexpr int OFF_LIMIT = OFF_BAR2 + 8;           // completion-wait limit, device clock cycles
constexpr int OFF_TSLOT = OFF_LIMIT + 8;          // TMEM base address (tcgen05.alloc)
constexpr int OFF_ERR = OFF_TSLOT + 4;            // sticky: an MMA wait gave up
constexpr int OFF_SKIP = OFF_ERR + 4;             // self-test: completion commits left out
constexpr int BYTES = (OFF_SKIP + 4 + 15) / 16 * 16;
static_assert(OFF_BAR % 8 == 0 && OFF_LIMIT % 8 == 0 && BYTES % 16 == 0, "tensor-core area layout");

// Default limit of a completion wait: about a second of device clock.
constexpr long long kWaitLimit = 2000000000ll;

__host__ __device__ constexpr size_t smem_bytes() { return (size_t)BYTES; }

}  // namespace tc
}  // namespace rgf

// The block's dynamic shared memory (every extern __shared__ array aliases it).
extern __shared__ __align__(1024) unsigned char rgf_dyn_smem[];

namespace rgf {
namespace tc {

__device__ __forceinline__ uint32_t su32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Byte offset of a shared-memory pointer from the start of dynamic shared memory.
__device__ __forceinline__ int dyn_off(const void* p) { return (int)(su32(p) - su32(rgf_dyn_smem)); }

// The tensor-core area, `off` bytes into dynamic shared memory.  Passed by
// value (one integer); every accessor is a shared-memory address.
struct Area {
    int off;
    __device__ unsigned char* base() const { return rgf_dyn_smem + off; }
    __device__ __nv_bfloat16* a() const { return reinterpret_cast<__nv_bfloat16*>(base() + OFF_A); }
    __device__ __nv_bfloat16* b() const { return reinterpret_cast<__nv_bfloat16*>(base() + OFF_B); }
    __device__ float* rsc() const { return reinterpret_cast<float*>(base() + OFF_RSC); }
    __device__ float* rfac() const { return reinterpret_cast<float*>(base() + OFF_RFAC); }
    __device__ float* csc() const { return reinterpret_cast<float*>(base() + OFF_CSC); }
    __device__ float* cfac() const { return reinterpret_cast<float*>(base() + OFF_CFAC); }
    __device__ unsigned* cmax() const { return reinterpret_cast<unsigned*>(base() + OFF_CMAX); }
    __device__ unsigned long long* bar() const { return reinterpret_cast<unsigned long long*>(base() + OFF_BAR); }
    __device__ unsigned long long* bar2() const { return reinterpret_cast<unsigned long long*>(base() + OFF_BAR2); }
    __device__ long long* limit() const { return reinterpret_cast<long long*>(base() + OFF_LIMIT); }
    __device__ int* skip() const { return reinterpret_cast<int*>(base() + OFF_SKIP); }
    __device__ uint32_t* tslot() const { return reinterpret_cast<uint32_t*>(base() + OFF_TSLOT); }
    __device__ int* err() const { return reinterpret_cast<int*>(base() + OFF_ERR); }
};

// The area plus the mbarrier phase this thread expects next (every thread
// waits on every commit, so every thread tracks the same phase).
struct State {
    Area ar;
    uint32_t phase;
};

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
// 32 lanes x 4 consecutive columns of TMEM.
__device__ __forceinline__ void ld4(uint32_t addr, float* v) {
    uint32_t r[4];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Allocates all 512 TMEM columns (warp 0) and initialises the mbarriers, the
// completion-wait limit and the self-test switch (skip != 0: the completion of
// the MMAs is never committed, so the first wait runs into its limit).  Must
// be called by every thread of the block (it ends with a barrier); the block
// must be the only one on its SM that uses TMEM.  Returns the initial phase.
__device__ inline uint32_t setup(Area ar, long long limit = kWaitLimit, int skip = 0) {
    if ((threadIdx.x >> 5) == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;"
                     :: "r"(su32(ar.tslot())) : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(ar.bar())) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(su32(ar.bar2())) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *ar.err() = 0;
        *ar.limit() = limit;
        *ar.skip() = skip;
    }
    fence_before();
    __syncthreads();
    fence_after();
    return 0u;
}

// Releases TMEM.  Every thread.  If a completion wait gave up, MMAs may still
// be in flight: the issuing thread commits them to the second mbarrier and the
// block waits for it (bounded by the default limit) before the release.
__device__ inline void teardown(Area ar) {
    fence_before();
    __syncthreads();
    if (*(volatile int*)ar.err()) {
        if (threadIdx.x == 0)
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                         :: "r"(su32(ar.bar2())) : "memory");
        const long long t0 = clock64();
        while (!try_wait(ar.bar2(), 0u) && clock64() - t0 <= kWaitLimit) {
        }
        fence_after();
        fence_before();
        __syncthreads();
    }
    if ((threadIdx.x >> 5) == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" :: "r"(*ar.tslot()) : "memory");
}

// Waits (every thread) for the MMAs committed last; gives up after the
// block's limit (about a second of device clock by default) and sets the
// sticky error flag, after which later waits return at once.  Returns the next
// phase.
__device__ inline uint32_t wait_mma(Area ar, uint32_t phase) {
    if (!*(volatile int*)ar.err()) {
        bool done = try_wait(ar.bar(), phase);
        if (!done) {
            const long long t0 = clock64(), lim = *(volatile long long*)ar.limit();
            while (!done) {
                done = try_wait(ar.bar(), phase);
                if (!done && clock64() - t0 > lim) break;
            }
            if (!done) *(volatile int*)ar.err() = 1;
        }
    }
    fence_after();
    return phase ^ 1u;
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

// Slicing scale 2^(7-e) and output factor 2^(e-7) for a row / column maximum
// mx, with e the least integer such that mx < 2^e (from the exponent field:
// mx in [2^(E-127), 2^(E-126)) for a normal binary32 with biased exponent E).
__device__ __forceinline__ void scales(float mx, float& sc, float& fac) {
    const unsigned E = (__float_as_uint(mx) >> 23) & 0xFFu;
    if (!(mx <= 3.0e38f)) {          // NaN or Inf: poison the outputs of this row / column
        sc = 1.0f;
        fac = __int_as_float(0x7fc00000);
    } else if (E < 27u) {            // below 2^-100 (zeros, subnormals): treat as zero
        sc = 0.0f;
        fac = 0.0f;
    } else {
        const int e = (int)E - 126;
        sc = __int_as_float((134 - e) << 23);
        fac = __int_as_float((120 + e) << 23);
    }
}

// ---------------------------------------------------------------------------
// Binary64 operands (accessors with kF64 = true).  The scale of a row / column
// comes from the largest binary64 exponent field in it, and the digits of a
// value from its 53-bit integer significand: integer arithmetic only, no work
// on the FP64 pipe.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned exp64(double v) {
    return (unsigned)((unsigned long long)__double_as_longlong(v) >> 52) & 0x7FFu;
}

// Slicing scale 2^(7-e) and output factor 2^(e-7) for a largest biased
// binary64 exponent E (values below 2^(E-1022) in magnitude): e = E - 1022.
// E = 2047 (NaN, Inf) and e > 126 (beyond binary32) poison the outputs;
// below 2^-100 the row / column counts as zero -- as scales() does.
__device__ __forceinline__ void scales64(unsigned E, float& sc, float& fac) {
    const int e = (int)E - 1022;
    if (E == 2047u || e > 126) {
        sc = 1.0f;
        fac = __int_as_float(0x7fc00000);
    } else if (e < -99) {
        sc = 0.0f;
        fac = 0.0f;
    } else {
        sc = __int_as_float((134 - e) << 23);
        fac = __int_as_float((120 + e) << 23);
    }
}

// The S signed base-256 digits of the binary64 value v times the slicing scale
// sc = 2^(7-e) (|v| < 2^e): X = round(v 2^(55-e)) from the significand by a
// shift (|X| < 2^55), then balanced digits from the lowest up,
//     d_i in [-128, 127] (d_0 in [-128, 128]),  v sc ~ sum_i d_i 2^(-8 i),
// the rounding of X being the only error (half a unit of 2^(-48) of sc's unit,
// below the lowest digit).  Zero / subnormal v, or sc = 0, give zero digits.
__device__ __forceinline__ void digits64(double v, float sc, float* d) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7FFull);
    const unsigned scb = __float_as_uint(sc);
    long long X = 0;
    if (E != 0 && E != 2047 && (scb & 0x7F800000u) != 0u) {
        const int e = 134 - (int)((scb >> 23) & 0xFFu);
        const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
        const int sh = E - 1020 - e;              // X = M 2^sh, sh <= 2
        unsigned long long mag = 0;
        if (sh >= 0) mag = M << sh;
        else if (sh > -60) mag = (M + (1ull << (-sh - 1))) >> (-sh);
        X = (b >> 63) ? -(long long)mag : (long long)mag;
    }
#pragma unroll
    for (int i = S - 1; i >= 1; --i) {
        const long long r = ((X + 128) & 255) - 128;
        d[i] = (float)r;
        X = (X - r) >> 8;                         // exact: X - r is a multiple of 256
    }
    d[0] = (float)X;
}

// Whether an accessor works on binary64 (kF64 = true) or double-float values.
template <class T, class = void>
struct IsF64 : std::false_type {};
template <class T>
struct IsF64<T, std::void_t<decltype(T::kF64)>> : std::integral_constant<bool, T::kF64> {};

// C op= A B, A: M x Kc (M <= 128), B: Kc x N, complex double-float, through the
// accessor object `op` (passed by value):
//   zf op.a(m, k), op.b(k, n)                 operand entries
//   bool op.colA()                            true when a(m, k) is contiguous in m
//   Op::Old op.load(m, n, first)              the target of (m, n) before the
//                                             update (issued before the last MMA
//                                             wait, so its latency overlaps it)
//   void op.store(m, n, old, re, im, first)   writes the target from old and
//                                             (A B)[m][n] = re + i im over one group
//                                             of up to 96 inner entries; first =
//                                             the first group
// With Op::kF64 = true the entries are binary64 (zd), sliced by digits64, and
// store receives re, im in binary64: the six accumulators are summed
// error-free in binary32 to three terms s + t + w (|w| < 2^-40 |s|), which are
// added in binary64 -- a product accurate to a few units of 2^-53 of (row max
// x column max x inner dimension).
// Called by every thread of the block (NT = 512); ends with a barrier.
// Returns the next mbarrier phase.
template <class Op>
__device__ __forceinline__ uint32_t zgemm(Op op, int M, int N, int Kc, Area ar, uint32_t phase) {
    static_assert(NT == 512, "zgemm assumes 512 threads");
    constexpr bool F64 = IsF64<Op>::value;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t tmem = *ar.tslot();
    float* rsc = ar.rsc();
    float* rfac = ar.rfac();
    float* csc = ar.csc();
    float* cfac = ar.cfac();
    unsigned* cmax = ar.cmax();
    __nv_bfloat16* ta0 = ar.a();
    __nv_bfloat16* tb = ar.b();
    const int q4 = warp & 3, mrow = 32 * q4 + lane, cgrp = warp >> 2;   // drain mapping
    for (int g0 = 0; g0 < Kc; g0 += KGRP) {
        const int kg = min(KGRP, Kc - g0);
        const int nch = (kg + KCH - 1) / KCH;
        const bool cacheA = nch <= NCA;
        // row scales over this group
        const bool colA = op.colA();
        if constexpr (F64) {
            if (colA) {
                if (tid < 128) {
                    unsigned mx = 0u;
                    if (tid < M)
                        for (int k = 0; k < kg; ++k) {
                            const zd v = op.a(tid, g0 + k);
                            mx = max(mx, max(exp64(v.re), exp64(v.im)));
                        }
                    scales64(mx, rsc[tid], rfac[tid]);
                }
            } else {
                for (int m = warp; m < 128; m += NWARP) {
                    unsigned mx = 0u;
                    if (m < M)
                        for (int k = lane; k < kg; k += 32) {
                            const zd v = op.a(m, g0 + k);
                            mx = max(mx, max(exp64(v.re), exp64(v.im)));
                        }
                    mx = __reduce_max_sync(0xffffffffu, mx);
                    if (lane == 0) scales64(mx, rsc[m], rfac[m]);
                }
            }
        } else if (colA) {
            if (tid < 128) {
                float mx = 0.0f;
                if (tid < M)
                    for (int k = 0; k < kg; ++k) {
                        const zf v = op.a(tid, g0 + k);
                        mx = nmax(mx, nmax(fabsf(v.re.hi), fabsf(v.im.hi)));
                    }
                scales(mx, rsc[tid], rfac[tid]);
            }
        } else {
            for (int m = warp; m < 128; m += NWARP) {
                float mx = 0.0f;
                if (m < M)
                    for (int k = lane; k < kg; k += 32) {
                        const zf v = op.a(m, g0 + k);
                        mx = nmax(mx, nmax(fabsf(v.re.hi), fabsf(v.im.hi)));
                    }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mx = nmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (lane == 0) scales(mx, rsc[m], rfac[m]);
            }
        }
        for (int n0 = 0; n0 < N; n0 += MAXC) {
            const int nc = min(MAXC, N - n0);
            const int ncp = (nc + 7) & ~7;
            const int NR = 2 * ncp;               // real output columns (Re, Im interleaved)
            if (tid < MAXC) cmax[tid] = 0u;
            __syncthreads();
            if (tid < (NT / MAXC) * MAXC) {
                const int c = tid % MAXC, ks = tid / MAXC;
                float mx = 0.0f;
                if constexpr (F64) {
                    unsigned ex = 0u;
                    if (c < nc)
                        for (int k = ks; k < kg; k += NT / MAXC) {
                            const zd v = op.b(g0 + k, n0 + c);
                            ex = max(ex, max(exp64(v.re), exp64(v.im)));
                        }
                    if (c < nc) atomicMax(&cmax[c], ex);
                } else {
                    if (c < nc)
                        for (int k = ks; k < kg; k += NT / MAXC) {
                            const zf v = op.b(g0 + k, n0 + c);
                            mx = nmax(mx, nmax(fabsf(v.re.hi), fabsf(v.im.hi)));
                        }
                    if (c < nc) atomicMax(&cmax[c], __float_as_uint(mx));
                }
            }
            __syncthreads();
            if (tid < MAXC) {
                if constexpr (F64) scales64(cmax[tid], csc[tid], cfac[tid]);
                else scales(__uint_as_float(cmax[tid]), csc[tid], cfac[tid]);
            }
            __syncthreads();
            typename Op::Old old[4];
            uint32_t init = 0u;
            for (int ch = 0; ch < nch; ++ch) {
                const int k0 = ch * KCH;
                __nv_bfloat16* ta = ta0 + (cacheA ? ch : 0) * (S * TILE);
                if (!cacheA || n0 == 0) {
                    // A': 128 rows x 8 complex entries, two per thread
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int e = tid + h * NT;
                        const int m = colA ? (e & 127) : (e >> 3);
                        const int k = colA ? (e >> 7) : (e & 7);
                        float dr[S], di[S];
                        if (m < M && k0 + k < kg) {
                            const float sc = rsc[m];
                            if constexpr (F64) {
                                const zd v = op.a(m, g0 + k0 + k);
                                digits64(v.re, sc, dr);
                                digits64(v.im, sc, di);
                            } else {
                                const zf v = op.a(m, g0 + k0 + k);
                                digits(v.re.hi, v.re.lo, sc, dr);
                                digits(v.im.hi, v.im.lo, sc, di);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < S; ++i) { dr[i] = 0.0f; di[i] = 0.0f; }
                        }
                        const int o = tile_off(m, 2 * k);
#pragma unroll
                        for (int i = 0; i < S; ++i) {
                            const float w = dweight(i);
                            *reinterpret_cast<__nv_bfloat162*>(ta + i * TILE + o) =
                                __floats2bfloat162_rn(dr[i] * w, di[i] * w);
                        }
                    }
                }
                // B': 8 complex entries x ncp columns, one per thread
                {
                    const int k = tid >> 6, c = tid & 63;
                    if (c < ncp) {
                        float dr[S], di[S];
                        if (c < nc && k0 + k < kg) {
                            const float sc = csc[c];
                            if constexpr (F64) {
                                const zd v = op.b(g0 + k0 + k, n0 + c);
                                digits64(v.re, sc, dr);
                                digits64(v.im, sc, di);
                            } else {
                                const zf v = op.b(g0 + k0 + k, n0 + c);
                                digits(v.re.hi, v.re.lo, sc, dr);
                                digits(v.im.hi, v.im.lo, sc, di);
                            }
                        } else {
#pragma unroll
                            for (int i = 0; i < S; ++i) { dr[i] = 0.0f; di[i] = 0.0f; }
                        }
                        const int ore = tile_off(2 * c, 2 * k), oim = tile_off(2 * c + 1, 2 * k);
#pragma unroll
                        for (int i = 0; i < S; ++i) {
                            const float w = dweight(i);
                            *reinterpret_cast<__nv_bfloat162*>(tb + i * TILE + ore) =
                                __floats2bfloat162_rn(dr[i] * w, -di[i] * w);
                            *reinterpret_cast<__nv_bfloat162*>(tb + i * TILE + oim) =
                                __floats2bfloat162_rn(di[i] * w, dr[i] * w);
                        }
                    }
                }
                fence_async_smem();
                __syncthreads();
                if (tid == 0) {
                    fence_after();
                    const uint32_t id = idesc(NR);
                    // digit tile i starts TILE * 2 bytes after tile i - 1: its
                    // descriptor's address field (16-byte units, every shared
                    // address below 2^18) is kTileDesc further on
                    constexpr uint64_t kTileDesc = (uint64_t)(TILE * 2) >> 4;
                    const uint64_t da = sdesc(ta), db = sdesc(tb);
#pragma unroll
                    for (int l = 0; l < S; ++l)
#pragma unroll
                        for (int i = 0; i <= l; ++i) {
                            const int j = l - i, acc = l < NACC - 1 ? l : NACC - 1;
                            mma(tmem + (uint32_t)(ACOLS * acc), da + (uint64_t)i * kTileDesc,
                                db + (uint64_t)j * kTileDesc, id, (init >> acc) & 1u);
                            init |= 1u << acc;
                        }
                    if (!*ar.skip()) commit(ar.bar());
                }
                if (ch == nch - 1 && mrow < M) {
                    // targets of this thread's first drain block, loaded under
                    // the last MMAs
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int c = 4 * cgrp + j;
                        if (c < nc) old[j] = op.load(mrow, n0 + c, g0 == 0);
                    }
                }
                phase = wait_mma(ar, phase);   // tiles may be rewritten; accumulators final
                init = (1u << NACC) - 1u;
            }
            // drain: warp w reads lanes 32 (w & 3) .. +31 (rows) and the 8-column
            // blocks (4 complex columns) w >> 2, + 4, + 8; each block's targets
            // are loaded before its TMEM reads
            {
                const float rf = rfac[mrow];
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int cb = cgrp + 4 * b;
                    if (cb < NR / 8) {
                        if (b > 0 && mrow < M) {
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const int c = 4 * cb + j;
                                if (c < nc) old[j] = op.load(mrow, n0 + c, g0 == 0);
                            }
                        }
                        const uint32_t ad = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(8 * cb);
                        // two halves of 4 columns (2 complex columns); levels
                        // 0 + 1 and 2 + 3 pair up error-free, 4 + 5 in binary32
                        // (below 2^-32 of the scale), then one double-float sum
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const uint32_t ah = ad + 4u * h;
                            float a0[4], a1[4], a2[4], a3[4], a4[4], a5[4];
                            ld4(ah, a0);
                            ld4(ah + ACOLS, a1);
                            ld4(ah + 2 * ACOLS, a2);
                            ld4(ah + 3 * ACOLS, a3);
                            ld4(ah + 4 * ACOLS, a4);
                            ld4(ah + 5 * ACOLS, a5);
                            ld_wait();
                            if constexpr (F64) {
                                // s + t + w exactly up to the rounding of w
                                // (below 2^-70 of s), then binary64
                                double z[4];
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    float s01, e01, s23, e23, r45, e45, s, e, p, pe, q, qe, t, te;
                                    two_sum(a0[j], a1[j], s01, e01);
                                    two_sum(a2[j], a3[j], s23, e23);
                                    two_sum(a4[j], a5[j], r45, e45);
                                    two_sum(s01, s23, s, e);
                                    two_sum(e01, e, p, pe);
                                    two_sum(e23, r45, q, qe);
                                    two_sum(p, q, t, te);
                                    const float w = __fadd_rn(__fadd_rn(pe, qe), __fadd_rn(te, e45));
                                    z[j] = (double)s + ((double)t + (double)w);
                                }
                                if (mrow < M) {
#pragma unroll
                                    for (int jj = 0; jj < 2; ++jj) {
                                        const int j = 2 * h + jj, c = 4 * cb + j;
                                        if (c < nc) {
                                            const double f = (double)rf * (double)cfac[c];
                                            op.store(mrow, n0 + c, old[j], z[2 * jj] * f, z[2 * jj + 1] * f,
                                                     g0 == 0);
                                        }
                                    }
                                }
                            } else {
                                float hi[4], lo[4];
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    float s01, e01, s23, e23, s, e;
                                    two_sum(a0[j], a1[j], s01, e01);        // exact
                                    two_sum(a2[j], a3[j], s23, e23);        // exact
                                    const float r45 = __fadd_rn(a4[j], a5[j]);
                                    two_sum(s01, s23, s, e);
                                    fast_two_sum(s, __fadd_rn(__fadd_rn(e01, e), __fadd_rn(e23, r45)), hi[j], lo[j]);
                                }
                                if (mrow < M) {
#pragma unroll
                                    for (int jj = 0; jj < 2; ++jj) {
                                        const int j = 2 * h + jj, c = 4 * cb + j;
                                        if (c < nc) {
                                            const float f = rf * cfac[c];
                                            const df32 re{__fmul_rn(hi[2 * jj], f), __fmul_rn(lo[2 * jj], f)};
                                            const df32 im{__fmul_rn(hi[2 * jj + 1], f), __fmul_rn(lo[2 * jj + 1], f)};
                                            op.store(mrow, n0 + c, old[j], re, im, g0 == 0);
                                        }
                                    }
                                }
                            }
                        }
                    }
                }
            }
            fence_before();
            __syncthreads();            // accumulators read; next pass may overwrite
        }
    }
    return phase;
}

}  // namespace tc
}  // namespace rgf
