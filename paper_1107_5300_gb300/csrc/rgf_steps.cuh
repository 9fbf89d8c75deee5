// rgf_steps.cuh -- one column step of the forward RGF recursion (Eqs. 4-5) and
// the helpers shared by the forward sweep (rgf_half.cuh) and the gradient sweep
// (rgf_grad.cu).  See rgf_half.cuh for the column slicing.
#pragma once

#include <type_traits>

#include "rgf_device.cuh"
#include "rgf_internal.h"

namespace rgf {

template <class R>
struct SweepSmem {
    GJSmem<R> gj;
    cx<R>* gemm;
    uint8_t* kc;     // keep mask of the current column
    uint8_t* kp;     // keep mask of the previous column
    uint8_t* kn;     // keep mask of the next column (gradient; second column of a pair)
    double* eps;
    double* red;
    tc::State* tcs;  // tensor-core state for the strip product, or nullptr
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

// Shared-memory layout of the sweep for a largest column size Kmax and panel
// width bm: the sweep's own buffers, then (with tc) the tensor-core area at the
// next 1024-byte boundary.  With tc the staging tiles of the binary64 GEMM
// (used only by the trace, after the last MMA) alias the tensor-core tiles.
__host__ __device__ inline size_t sweep_base_bytes(int Kmax, int bm, bool tc) {
    size_t b = 0;
    b += 4 * align16((size_t)Kmax * bm * 16);   // 2 panels, multipliers, pivot rows
    b += align16((size_t)bm * 16);              // pivot reciprocals
    if (!tc) b += align16(2 * 8 * 64 * 16);     // gemm tiles
    b += align16((size_t)Kmax * 8);             // eps
    b += align16(NWARP * 8);                    // red
    b += align16((size_t)Kmax * 4) * 2;         // perm, idx
    b += align16((size_t)(2 * bm + 1) * 4);     // displaced rows of a panel
    b += align16(16);                           // ctl
    b += align16(32);                           // pivot keys
    b += align16((size_t)Kmax) * 3;             // kc, kp, kn
    return b;
}
__host__ __device__ inline size_t tc_area_offset(int Kmax, int bm) {
    return (sweep_base_bytes(Kmax, bm, true) + 1023) & ~(size_t)1023;
}
__host__ __device__ inline size_t sweep_total_bytes(int Kmax, int bm, bool tc) {
    return tc ? tc_area_offset(Kmax, bm) + tc::smem_bytes() : sweep_base_bytes(Kmax, bm, false);
}
// The binary64 staging tiles (the only part of a binary64 layout beyond the
// tensor-core layout's own buffers) fit inside the digit tiles of A.
static_assert(2 * 8 * 64 * 16 + 1024 <= tc::OFF_B, "binary64 layout inside the tensor-core tiles");

// Panel width of the blocked Gauss-Jordan for a largest column size Kmax:
// the widest of 16, 8, 4, 2 whose layout fits the 227 KB of shared memory a
// block may use.
__host__ __device__ inline int gj_panel_width(int Kmax, bool tc = false) {
    int b = 16;
    while (b > 2 && sweep_total_bytes(Kmax, b, tc) > 232448) b >>= 1;
    return b;
}

// The layout for panel width bm (0: gj_panel_width(Kmax, tc)).  A binary64
// layout (tc false) carved with the panel width of a tensor-core launch ends
// inside that launch's digit tiles (its GEMM staging tiles are the only part
// past the sweep's own buffers), so a persistent block can alternate between
// the two without touching its mbarriers or TMEM address.
template <class R>
__device__ SweepSmem<R> carve(unsigned char* base, int Kmax, bool tc = false, int bm = 0) {
    SweepSmem<R> s;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
    if (bm <= 0) bm = gj_panel_width(Kmax, tc);
    s.gj.tcs = nullptr;
    s.tcs = nullptr;
    s.gj.bmax = bm;
    s.gj.panel = (cx<R>*)take((size_t)Kmax * bm * 16);
    s.gj.panel2 = (cx<R>*)take((size_t)Kmax * bm * 16);
    s.gj.mult = (cx<R>*)take((size_t)Kmax * bm * 16);
    s.gj.xrow = (cx<R>*)take((size_t)Kmax * bm * 16);
    s.gj.pinv = (cx<R>*)take((size_t)bm * 16);
    s.gemm = tc ? (cx<R>*)(base + tc_area_offset(Kmax, bm)) : (cx<R>*)take(2 * 8 * 64 * 16);
    s.eps = (double*)take((size_t)Kmax * 8);
    s.red = (double*)take(NWARP * 8);
    s.gj.perm = (int*)take((size_t)Kmax * 4);
    s.gj.idx = (int*)take((size_t)Kmax * 4);
    s.gj.pm = (int*)take((size_t)(2 * bm + 1) * 4);
    s.gj.ctl = (int*)take(16);
    s.gj.key = (unsigned long long*)take(32);
    s.kc = (uint8_t*)take((size_t)Kmax);
    s.kp = (uint8_t*)take((size_t)Kmax);
    s.kn = (uint8_t*)take((size_t)Kmax);
    return s;
}

// Sets up the tensor-core area behind the sweep's shared memory (TMEM
// allocation, mbarrier; every thread) and points the contractions at it.
template <class R>
__device__ void tc_attach(int Kmax, SweepSmem<R>& s, tc::State& st) {
    st.ar = tc::Area{(int)tc_area_offset(Kmax, gj_panel_width(Kmax, true))};
    st.phase = tc::setup(st.ar);
    s.gj.tcs = &st;
    s.tcs = &st;
}

// C (M x N) = op(A) (M x Kd) B (Kd x N), op(A) = A or A^T (ta; no
// conjugation), as a tensor-core product over one tile of up to 128 rows of C.
// C must not overlap A or B.
struct DenseOp {
    const zf* A;
    int lda;
    const zf* B;
    int ldb;
    zf* C;
    int ldc, r0;
    bool ta;
    using Old = float4;
    __device__ bool colA() const { return ta; }
    __device__ zf a(int m, int k) const {
        return ta ? A[(size_t)k * lda + r0 + m] : A[(size_t)(r0 + m) * lda + k];
    }
    __device__ zf b(int k, int n) const { return B[(size_t)k * ldb + n]; }
    __device__ float4 load(int m, int n, bool first) const {
        return first ? make_float4(0.f, 0.f, 0.f, 0.f)
                     : *reinterpret_cast<const float4*>(C + (size_t)(r0 + m) * ldc + n);
    }
    __device__ void store(int m, int n, float4 x, df32 re, df32 im, bool first) const {
        if (!first) {
            re = df_add(df32{x.x, x.y}, re);
            im = df_add(df32{x.z, x.w}, im);
        }
        *reinterpret_cast<float4*>(C + (size_t)(r0 + m) * ldc + n) = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
};

// The same product on binary64 operands (RGF_FP64_TC).
struct DenseOp64 {
    static constexpr bool kF64 = true;
    const zd* A;
    int lda;
    const zd* B;
    int ldb;
    zd* C;
    int ldc, r0;
    bool ta;
    using Old = zd;
    __device__ bool colA() const { return ta; }
    __device__ zd a(int m, int k) const {
        return ta ? A[(size_t)k * lda + r0 + m] : A[(size_t)(r0 + m) * lda + k];
    }
    __device__ zd b(int k, int n) const { return B[(size_t)k * ldb + n]; }
    __device__ zd load(int m, int n, bool first) const {
        return first ? zd{0.0, 0.0} : C[(size_t)(r0 + m) * ldc + n];
    }
    __device__ void store(int m, int n, zd x, double re, double im, bool first) const {
        C[(size_t)(r0 + m) * ldc + n] = first ? zd{re, im} : zd{x.re + re, x.im + im};
    }
};

// C = op(A) B on the tensor cores over row tiles of 128; one out-of-line copy
// for the gradient's dense products (arguments by value; the sweep's strip
// product is inlined).  Returns the next mbarrier phase.
static __device__ __noinline__ uint32_t tc_dense(int m, int n, int kd, const zf* A, int lda,
                                                 const zf* B, int ldb, zf* C, int ldc, bool ta,
                                                 tc::Area ar, uint32_t phase) {
    for (int r0 = 0; r0 < m; r0 += 128) {
        const DenseOp op{A, lda, B, ldb, C, ldc, r0, ta};
        phase = tc::zgemm(op, min(128, m - r0), n, kd, ar, phase);
    }
    return phase;
}

// The binary64 copy (RGF_FP64_TC's gradient products).
static __device__ __noinline__ uint32_t tc_dense64(int m, int n, int kd, const zd* A, int lda,
                                                   const zd* B, int ldb, zd* C, int ldc, bool ta,
                                                   tc::Area ar, uint32_t phase) {
    for (int r0 = 0; r0 < m; r0 += 128) {
        const DenseOp64 op{A, lda, B, ldb, C, ldc, r0, ta};
        phase = tc::zgemm(op, min(128, m - r0), n, kd, ar, phase);
    }
    return phase;
}

// C = op(A) B on the tensor cores when the block holds them (double-float
// operands; binary64 with TC64), else on the FP32 / FP64 pipes.  Every
// thread; ends with a barrier.
template <class R, bool TA, bool TC64 = false>
__device__ void dense_product(int m, int n, int kd, const cx<R>* A, int lda, const cx<R>* B, int ldb,
                              cx<R>* C, int ldc, SweepSmem<R>& s) {
    if constexpr (std::is_same<R, df32>::value) {
        if (s.tcs) {
            if (m <= 0 || n <= 0 || kd <= 0) {
                __syncthreads();
                return;
            }
            s.tcs->phase = tc_dense(m, n, kd, A, lda, B, ldb, C, ldc, TA, s.tcs->ar, s.tcs->phase);
            return;
        }
    } else if constexpr (std::is_same<R, double>::value && TC64) {
        if (s.tcs) {
            if (m <= 0 || n <= 0 || kd <= 0) {
                __syncthreads();
                return;
            }
            s.tcs->phase = tc_dense64(m, n, kd, A, lda, B, ldb, C, ldc, TA, s.tcs->ar, s.tcs->phase);
            return;
        }
    }
    cta_gemm<R, TA, false>(m, n, kd, A, lda, B, ldb, C, ldc, GEMM_SET, s.gemm);
}

// Everything a block needs to know about its chain.  dir: the direction of
// the column recursion this block runs -- 0 from the left lead (column k
// follows k - 1), 1 from the right lead (column k follows k + 1).
struct ChainCtx {
    const double* eps;
    const uint8_t* rem;
    int N, L, M, KL, KR, ncol, dir;
    double t, t2;
    df32 tf, t2f;    // t and t^2 in double-float, converted once
    zd z;
    const zd* lead;  // this chain's lead output (layout of LeadDev::off)
    // site basis of the lead-attached columns, the mode vectors (real parts)
    // and w_p = tau_p^2 g_p, located from `lead` on use (fewer live registers)
    __device__ const zd* SigL() const { return lead; }
    __device__ const zd* SigR() const { return lead + (size_t)KL * KL; }
    __device__ const zd* GamL() const { return SigR() + (size_t)KR * KR; }
    __device__ const zd* GamR() const { return GamL() + (size_t)KL * KL; }
    __device__ const zd* UL() const { return GamR() + (size_t)KR * KR; }
    __device__ const zd* UR() const { return UL() + (size_t)KL * KL; }
    __device__ const zd* w() const { return UR() + (size_t)KR * KR; }
};

__device__ inline ChainCtx make_ctx(const ChainDev& ch, const LeadDev& ld, const zd* leadout,
                                    double eta_d, int dir = 0) {
    ChainCtx c;
    c.eps = ch.eps;
    c.rem = ch.rem;
    c.N = ch.N;
    c.L = ch.L;
    c.M = 2 * ch.N;
    c.KL = col_KL(ch.N);
    c.KR = col_KR(ch.N);
    c.ncol = 4 * ch.L;
    c.dir = dir;
    c.t = ch.t;
    c.t2 = ch.t * ch.t;
    c.tf = df_from_double(c.t);
    c.t2f = df_from_double(c.t2);
    c.z = {ch.E, eta_d};
    c.lead = leadout + ld.off;
    return c;
}

// The hopping t and t^2 in the working precision.
template <class R> struct Hop;
template <> struct Hop<double> {
    static __device__ __forceinline__ double t(const ChainCtx& c) { return c.t; }
    static __device__ __forceinline__ double t2(const ChainCtx& c) { return c.t2; }
};
template <> struct Hop<df32> {
    static __device__ __forceinline__ df32 t(const ChainCtx& c) { return c.tf; }
    static __device__ __forceinline__ df32 t2(const ChainCtx& c) { return c.t2f; }
};

__device__ __forceinline__ int col_size(const ChainCtx& c, int k) { return ((k & 3) < 2) ? c.KL : c.KR; }

// Source stencil of the coupling W_k into column k (type c = k mod 4): entry i
// of column k is bonded to entries a0, a1 (-1 = none) of column k-1 (size Kp).
//   c = 1, 3: same row (t I);  c = 2: rows q, q+1 of the even column;
//   c = 0: rows p-1, p of the odd column of the previous cell.
__device__ __forceinline__ void col_src(int c, int i, int Kp, int& a0, int& a1) {
    if (c == 1 || c == 3) { a0 = i; a1 = -1; }
    else if (c == 2) { a0 = i; a1 = (i + 1 < Kp) ? i + 1 : -1; }
    else { a0 = i - 1; a1 = (i < Kp) ? i : -1; }
}
// Transposed stencil: entries b0, b1 of column k (size K) bonded to entry a of
// column k-1.
__device__ __forceinline__ void col_src_T(int c, int a, int K, int& b0, int& b1) {
    if (c == 1 || c == 3) { b0 = a; b1 = -1; }
    else if (c == 2) { b0 = (a - 1 >= 0 && a - 1 < K) ? a - 1 : -1; b1 = (a < K) ? a : -1; }
    else { b0 = (a < K) ? a : -1; b1 = (a + 1 < K) ? a + 1 : -1; }
}

// The column that precedes column k in the recursion of direction c.dir.
__device__ __forceinline__ int prev_col(const ChainCtx& c, int k) { return c.dir ? k + 1 : k - 1; }

// Entries a0, a1 (-1 = none) of the preceding column (size Kq) bonded to entry
// i of column k: the source stencil of W_k from the left, its transpose (the
// bonds of column k + 1 seen from column k) from the right.
__device__ __forceinline__ void prev_src(const ChainCtx& c, int k, int i, int Kq, int& a0, int& a1) {
    if (c.dir == 0) col_src(k & 3, i, Kq, a0, a1);
    else col_src_T((k + 1) & 3, i, Kq, a0, a1);
}

// Keep mask (0 = removed atom) and on-site energies of column k into shared memory.
__device__ inline void load_col(const ChainCtx& c, int k, uint8_t* km, double* eps) {
    if (k < 0 || k >= c.ncol) return;
    const int n = k >> 2, ct = k & 3, K = col_size(c, k);
    for (int i = threadIdx.x; i < K; i += NT) {
        size_t o = (size_t)n * c.M + 4 * i + ct;
        km[i] = c.rem ? (c.rem[o] == 0) : 1;
        if (eps) eps[i] = c.eps[o];
    }
}

template <class R>
__device__ __forceinline__ cx<R> ld_z(const zd* p) { return from_z<R>(p->re, p->im); }

// On-site energy of entry i of column k, and d_i = z - eps_i of a pair's
// second column (binary64 in, working precision out).
__device__ __forceinline__ double site_eps(const ChainCtx& c, int k, int i) {
    return c.eps[(size_t)(k >> 2) * c.M + 4 * i + (k & 3)];
}
template <class R>
__device__ __forceinline__ cx<R> pair_d(const ChainCtx& c, int kb, int i) {
    return from_z<R>(c.z.re - site_eps(c, kb, i), c.z.im);
}

// One interior step of a half's column recursion at column k (row-major,
// leading dimension KL), with q = prev_col(c, k) the column before it:
//   inv_column:   X = A_k = (z - eps_k) I - t^2 S^T g_q S (K x K; S the bond
//                 stencil between q and k, identity rows and columns at removed
//                 atoms), Gout = A_k^-1 (Gauss-Jordan; Gout may alias Gprev).
//                 Needs s.kc / s.eps of column k and s.kp of column q.  Returns
//                 the Gauss-Jordan flag.
//   strip_column: Y = Pprev W (R x K, R the rows of the half's corner block),
//                 Pout = Y Gk (Pout may alias Pprev; Y may alias the X of
//                 inv_column).  Needs s.kc and s.kp.
// The lead-attached first column of a half is prepared elsewhere (rgf_half.cuh).
// kb >= 0 (pair steps, kb = the pair's second column): the diagonal of X
// additionally loses t^2 kappa_i / d_i (see pair_scales; s.kn holds the keep
// mask of kb).
template <class R, bool TC64 = false>
__device__ int inv_column(const ChainCtx& c, int k, const cx<R>* Gprev, cx<R>* Gout, cx<R>* X,
                          SweepSmem<R>& s, int kb = -1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KL = c.KL, K = col_size(c, k), Kq = col_size(c, prev_col(c, k));
    double amax2 = 0.0;
    for (int i = warp; i < K; i += NWARP) {
        int a0, a1;
        prev_src(c, k, i, Kq, a0, a1);
        const bool ki = s.kc[i];
        const bool ka0 = a0 >= 0 && s.kp[a0], ka1 = a1 >= 0 && s.kp[a1];
        for (int l = lane; l < K; l += 32) {
            cx<R> v;
            if (!ki || !s.kc[l]) {
                v = (i == l) ? from_z<R>(1.0, 0.0) : czero<R>();
            } else {
                int b0, b1;
                prev_src(c, k, l, Kq, b0, b1);
                const bool kb0 = b0 >= 0 && s.kp[b0], kb1 = b1 >= 0 && s.kp[b1];
                cx<R> sig = czero<R>();
                if (ka0 && kb0) sig = cadd(sig, Gprev[(size_t)a0 * KL + b0]);
                if (ka0 && kb1) sig = cadd(sig, Gprev[(size_t)a0 * KL + b1]);
                if (ka1 && kb0) sig = cadd(sig, Gprev[(size_t)a1 * KL + b0]);
                if (ka1 && kb1) sig = cadd(sig, Gprev[(size_t)a1 * KL + b1]);
                sig = cscale(sig, Hop<R>::t2(c));
                v = (i == l) ? from_z<R>(c.z.re - s.eps[i], c.z.im) : czero<R>();
                if (kb >= 0 && i == l && s.kn[i])
                    v = csub(v, cscale(crecip(pair_d<R>(c, kb, i)), Hop<R>::t2(c)));
                v = csub(v, sig);
            }
            X[(size_t)i * KL + l] = v;
            const double a2 = (double)cabs2f(v);
            amax2 = (a2 > amax2 || isnan(a2)) ? a2 : amax2;
        }
    }
    amax2 = block_max(amax2, s.red);
    return cta_gj_invert<R, TC64>(X, K, KL, Gout, KL, s.gj, amax2);
}

template <class R, bool TC64 = false>
__device__ void strip_column(const ChainCtx& c, int k, const cx<R>* Gk, const cx<R>* Pprev,
                             cx<R>* Pout, cx<R>* Y, SweepSmem<R>& s, int nrows = -1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KL = c.KL, K = col_size(c, k), Kq = col_size(c, prev_col(c, k));
    const int rows = nrows >= 0 ? nrows : (c.dir ? c.KR : c.KL);
    for (int r = warp; r < rows; r += NWARP)
        for (int l = lane; l < K; l += 32) {
            cx<R> v = czero<R>();
            if (s.kc[l]) {
                int a0, a1;
                prev_src(c, k, l, Kq, a0, a1);
                if (a0 >= 0 && s.kp[a0]) v = cadd(v, Pprev[(size_t)r * KL + a0]);
                if (a1 >= 0 && s.kp[a1]) v = cadd(v, Pprev[(size_t)r * KL + a1]);
                v = cscale(v, Hop<R>::t(c));
            }
            Y[(size_t)r * KL + l] = v;
        }
    __syncthreads();                      // Y complete (Pprev no longer read)
    if constexpr (std::is_same<R, df32>::value) {
        if (s.tcs) {
            for (int r0 = 0; r0 < rows; r0 += 128) {
                const DenseOp op{Y, KL, Gk, KL, Pout, KL, r0, false};
                s.tcs->phase = tc::zgemm(op, min(128, rows - r0), K, K, s.tcs->ar, s.tcs->phase);
            }
            return;
        }
    } else if constexpr (std::is_same<R, double>::value && TC64) {
        if (s.tcs) {
            for (int r0 = 0; r0 < rows; r0 += 128) {
                const DenseOp64 op{Y, KL, Gk, KL, Pout, KL, r0, false};
                s.tcs->phase = tc::zgemm(op, min(128, rows - r0), K, K, s.tcs->ar, s.tcs->phase);
            }
            return;
        }
    }
    cta_gemm<R, false, false>(rows, K, K, Y, KL, Gk, KL, Pout, KL, GEMM_SET, s.gemm);
}

// C += A B^T (C: m x m, A and B: m x kd, leading dimension ld; C must not
// overlap A or B): the update of an interior domain's first-column block,
// G_aa += P_k Y^T.  On the tensor cores when the block holds them.
struct AccOp {
    const zf* A;
    const zf* B;
    zf* C;
    int ld, r0;
    using Old = float4;
    __device__ bool colA() const { return false; }
    __device__ zf a(int m, int k) const { return A[(size_t)(r0 + m) * ld + k]; }
    __device__ zf b(int k, int n) const { return B[(size_t)n * ld + k]; }
    __device__ float4 load(int m, int n, bool) const {
        return *reinterpret_cast<const float4*>(C + (size_t)(r0 + m) * ld + n);
    }
    __device__ void store(int m, int n, float4 x, df32 re, df32 im, bool) const {
        const df32 r = df_add(df32{x.x, x.y}, re), q = df_add(df32{x.z, x.w}, im);
        *reinterpret_cast<float4*>(C + (size_t)(r0 + m) * ld + n) = make_float4(r.hi, r.lo, q.hi, q.lo);
    }
};
struct AccOp64 {
    static constexpr bool kF64 = true;
    const zd* A;
    const zd* B;
    zd* C;
    int ld, r0;
    using Old = zd;
    __device__ bool colA() const { return false; }
    __device__ zd a(int m, int k) const { return A[(size_t)(r0 + m) * ld + k]; }
    __device__ zd b(int k, int n) const { return B[(size_t)n * ld + k]; }
    __device__ zd load(int m, int n, bool) const { return C[(size_t)(r0 + m) * ld + n]; }
    __device__ void store(int m, int n, zd x, double re, double im, bool) const {
        C[(size_t)(r0 + m) * ld + n] = zd{x.re + re, x.im + im};
    }
};

// Out-of-line copies (one each), so that the interior recursion carries no
// third inlined tensor-core product beside the inverse's and the strip's.
static __device__ __noinline__ uint32_t tc_acc(int m, int kd, const zf* A, const zf* B, zf* C, int ld,
                                               tc::Area ar, uint32_t phase) {
    for (int r0 = 0; r0 < m; r0 += 128) {
        const AccOp op{A, B, C, ld, r0};
        phase = tc::zgemm(op, min(128, m - r0), m, kd, ar, phase);
    }
    return phase;
}
static __device__ __noinline__ uint32_t tc_acc64(int m, int kd, const zd* A, const zd* B, zd* C,
                                                 int ld, tc::Area ar, uint32_t phase) {
    for (int r0 = 0; r0 < m; r0 += 128) {
        const AccOp64 op{A, B, C, ld, r0};
        phase = tc::zgemm(op, min(128, m - r0), m, kd, ar, phase);
    }
    return phase;
}

template <class R, bool TC64 = false>
__device__ void acc_product(int m, int kd, const cx<R>* A, const cx<R>* B, cx<R>* C, int ld,
                            SweepSmem<R>& s) {
    if constexpr (std::is_same<R, df32>::value) {
        if (s.tcs) {
            s.tcs->phase = tc_acc(m, kd, A, B, C, ld, s.tcs->ar, s.tcs->phase);
            return;
        }
    } else if constexpr (std::is_same<R, double>::value && TC64) {
        if (s.tcs) {
            s.tcs->phase = tc_acc64(m, kd, A, B, C, ld, s.tcs->ar, s.tcs->phase);
            return;
        }
    }
    cta_gemm<R, false, true>(m, m, kd, A, ld, B, ld, C, ld, GEMM_ADD, s.gemm);
}

// Two columns a, b = the next one in the recursion, joined by t I between the
// atoms of one row (the pairs c0-c1 and c2-c3 of a cell), in one inverse.
// Column b has no bond inside itself, so its slice matrix A_b = D - W g_a W
// (D = diag(d), d_i = z - eps_i for kept atoms and 1 for removed ones;
// W = t diag(kappa), kappa_i = both atoms of row i kept) is the Schur
// complement of the pair's block matrix [[X, -W], [-W, D]], X = A_a.  Taking
// the complement the other way round, with Z = (X - W D^-1 W)^-1,
//   g_b  = D^-1 + D^-1 W Z W D^-1 = diag(1/d) + diag(s) Z diag(s),
//   P_b  = P_q W_a G_ab = (P_q W_a) Z diag(s),      s_i = t kappa_i / d_i,
// so the pair costs one Gauss-Jordan inverse (of X with its diagonal shifted
// by -t s_i) and one strip product instead of two of each.  Used only when
// every kept atom of b has |d_i| >= kPairMinD (pair_ok): near an isolated-atom
// resonance 1/d grows and g_b's two terms cancel.  Needs s.kc / s.eps of a,
// s.kp of the column before a, s.kn / s.epsb of b.  On return G = g_b and
// P = P_b.  Returns the Gauss-Jordan flag.
constexpr double kPairMinD = 1e-4;   // eV

// Every thread: whether the pair whose second column is kb may be joined (no
// kept atom of kb within kPairMinD of E).  Needs s.kn.  Ends with a barrier.
template <class R>
__device__ bool pair_ok(const ChainCtx& c, int kb, SweepSmem<R>& s) {
    bool bad = false;
    for (int i = threadIdx.x; i < col_size(c, kb); i += NT) {
        if (s.kn[i]) {
            const double dr = c.z.re - site_eps(c, kb, i), dm = c.z.im;
            if (!(dr * dr + dm * dm >= kPairMinD * kPairMinD)) bad = true;
        }
    }
    return __syncthreads_or(bad) == 0;
}

// The two elementwise halves of a pair step around the strip product (the
// inverse of the shifted A_a is inv_column with kb): pair_scales sets up
// s_i and 1/d_i in the Gauss-Jordan scratch (free between inverses) and
// scales G = Z into Z diag(s); pair_finish turns it into
// g_b = diag(1/d) + diag(s) Z diag(s).  Every thread; barriers at the end.
template <class R>
__device__ void pair_scales(const ChainCtx& c, int ka, int kb, cx<R>* G, SweepSmem<R>& s) {
    const int KL = c.KL, K = col_size(c, ka);
    cx<R>* sc = s.gj.mult;
    cx<R>* di = s.gj.xrow;
    for (int i = threadIdx.x; i < K; i += NT) {
        if (s.kn[i]) {
            const cx<R> inv = crecip(pair_d<R>(c, kb, i));
            di[i] = inv;
            sc[i] = s.kc[i] ? cscale(inv, Hop<R>::t(c)) : czero<R>();
        } else {
            di[i] = from_z<R>(1.0, 0.0);
            sc[i] = czero<R>();
        }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += NT) {
        const int i = e / K, l = e - i * K;
        G[(size_t)i * KL + l] = cmul(G[(size_t)i * KL + l], sc[l]);
    }
    __syncthreads();
}

template <class R>
__device__ void pair_finish(const ChainCtx& c, int ka, cx<R>* G, SweepSmem<R>& s) {
    const int KL = c.KL, K = col_size(c, ka);
    const cx<R>* sc = s.gj.mult;
    const cx<R>* di = s.gj.xrow;
    for (int e = threadIdx.x; e < K * K; e += NT) {
        const int i = e / K, l = e - i * K;
        cx<R> v = cmul(sc[i], G[(size_t)i * KL + l]);
        if (i == l) v = cadd(v, di[i]);
        G[(size_t)i * KL + l] = v;
    }
    __syncthreads();
}

// Tr[Gamma_L P Gamma_R P^dagger] in binary64.  P: KL x KR (ld KL) in the working
// precision; Xs, Zs, Cz: KL x KL scratch (16-byte elements).
template <class R>
__device__ double trace_T(const ChainCtx& c, const cx<R>* P, cx<R>* Cz, cx<R>* Xs, cx<R>* Zs,
                          SweepSmem<R>& s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KL = c.KL, KR = c.KR;
    const zd* Pz;
    if (std::is_same<R, double>::value) {
        Pz = reinterpret_cast<const zd*>(P);
    } else {
        zd* w = reinterpret_cast<zd*>(Cz);
        for (int i = warp; i < KL; i += NWARP)
            for (int l = lane; l < KR; l += 32) w[(size_t)i * KL + l] = to_z(P[(size_t)i * KL + l]);
        __syncthreads();
        Pz = w;
    }
    zd* X = reinterpret_cast<zd*>(Xs);
    zd* Z = reinterpret_cast<zd*>(Zs);
    zd* gsm = reinterpret_cast<zd*>(s.gemm);
    cta_gemm<double, false, false>(KL, KR, KL, c.GamL(), KL, Pz, KL, X, KL, GEMM_SET, gsm);
    cta_gemm<double, false, false>(KL, KR, KR, Pz, KL, c.GamR(), KR, Z, KL, GEMM_SET, gsm);
    double acc = 0.0;
    for (int e = threadIdx.x; e < KL * KR; e += NT) {
        int a = e / KR, b = e % KR;
        zd x = X[(size_t)a * KL + b], zz = Z[(size_t)a * KL + b];
        acc += x.re * zz.re + x.im * zz.im;    // Re(x conj(z))
    }
    return block_sum(acc, s.red);
}

// Status word of a finished chain from the Gauss-Jordan flags and T.
__device__ inline int chain_status(const ChainCtx& c, int flag, double T) {
    const double nch = (double)channels(c.N, c.t, c.z.re);
    if (flag & 4) return ST_ETIMEOUT;
    if ((flag & 2) || !isfinite(T)) return ST_ENONFINITE;
    if (flag & 1) return ST_ESINGULAR;
    if (T < -1e-6 || T > nch + 1e-6) return ST_EBOUNDS;
    return ST_OK;
}

__device__ inline int lead_state(const int* lead_status, int lead) {
    int lst = lead_status[2 * lead];
    if (lst == ST_OK) lst = lead_status[2 * lead + 1];
    return lst;
}

}  // namespace rgf
