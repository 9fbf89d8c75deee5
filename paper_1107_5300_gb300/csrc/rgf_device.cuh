// rgf_device.cuh -- thread-block (CTA) level dense complex kernels used by the
// RGF sweeps: a tiled GEMM and an in-place Gauss-Jordan inverse with partial
// pivoting.  All matrices are row-major in global memory (L2-resident per
// chain); every routine is called by all threads of the block and ends with a
// __syncthreads().  The block size is RGF_NT threads.
#pragma once

#include <cooperative_groups.h>

#include <type_traits>

#include "rgf_common.cuh"
#include "rgf_tc.cuh"

namespace rgf {

// The blocks that share one chain: block `rank` of a cluster of C.  Work on
// columns (or rows) is split into C contiguous ranges; cl_sync() is a cluster
// barrier (a block barrier when C = 1).
struct Team {
    int rank, C;
    __device__ int lo(int n) const { return (int)(((long long)n * rank) / C); }
    __device__ int hi(int n) const { return (int)(((long long)n * (rank + 1)) / C); }
};
__device__ __forceinline__ void cl_sync(const Team& tm) {
    if (tm.C > 1) cooperative_groups::this_cluster().sync();
    else __syncthreads();
}

// Broadcast of lane 0's complex value across the warp.
__device__ __forceinline__ zd shfl0(zd v) {
    return {__shfl_sync(0xffffffffu, v.re, 0), __shfl_sync(0xffffffffu, v.im, 0)};
}
__device__ __forceinline__ zf shfl0(zf v) {
    return {{__shfl_sync(0xffffffffu, v.re.hi, 0), __shfl_sync(0xffffffffu, v.re.lo, 0)},
            {__shfl_sync(0xffffffffu, v.im.hi, 0), __shfl_sync(0xffffffffu, v.im.lo, 0)}};
}

// ---------------------------------------------------------------------------
// Block reductions
// ---------------------------------------------------------------------------
// Max of a non-negative binary64 value over the block; NaN wins (so that a
// non-finite matrix is noticed).  red: >= NWARP doubles of shared memory.
__device__ __forceinline__ double block_max(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (isnan(w) || w > v) ? w : v;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = red[0];
    for (int w = 1; w < NWARP; ++w) {
        double x = red[w];
        r = (isnan(x) || x > r) ? x : r;
    }
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    for (int w = 0; w < NWARP; ++w) r += red[w];
    __syncthreads();
    return r;
}

// ---------------------------------------------------------------------------
// C (m x n) {=, +=, -=} op(A) (m x kd) * op(B) (kd x n)
// op(X) = X or X^T (no conjugation).  64 x 64 output tiles, k-chunks of 8,
// each thread owns a 2 x 4 register tile.  C must not alias A or B.
// smem: 2 * 8 * 64 elements of cx<R>.
// ---------------------------------------------------------------------------
enum GemmMode { GEMM_SET = 0, GEMM_ADD = 1, GEMM_SUB = 2 };

template <class R, bool TA, bool TB>
__device__ void cta_gemm(int m, int n, int kd, const cx<R>* __restrict__ A, int lda,
                         const cx<R>* __restrict__ B, int ldb, cx<R>* __restrict__ C, int ldc,
                         int mode, cx<R>* sm) {
    cx<R>* As = sm;            // [8][64], k-major
    cx<R>* Bs = sm + 8 * 64;   // [8][64]
    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    static_assert(NT == 512, "cta_gemm assumes 512 threads");
    for (int i0 = 0; i0 < m; i0 += 64) {
        for (int j0 = 0; j0 < n; j0 += 64) {
            cx<R> acc[2][4];
#pragma unroll
            for (int r = 0; r < 2; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[r][c] = czero<R>();
            for (int k0 = 0; k0 < kd; k0 += 8) {
                {
                    int r, kk;
                    if (TA) { kk = tid >> 6; r = tid & 63; }   // A^T: rows of A are k
                    else    { r = tid >> 3;  kk = tid & 7;  }
                    int gi = i0 + r, gk = k0 + kk;
                    cx<R> v = czero<R>();
                    if (gi < m && gk < kd) v = TA ? A[(size_t)gk * lda + gi] : A[(size_t)gi * lda + gk];
                    As[kk * 64 + r] = v;
                }
                {
                    int kk, c;
                    if (TB) { c = tid >> 3; kk = tid & 7; }
                    else    { kk = tid >> 6; c = tid & 63; }
                    int gk = k0 + kk, gj = j0 + c;
                    cx<R> v = czero<R>();
                    if (gk < kd && gj < n) v = TB ? B[(size_t)gj * ldb + gk] : B[(size_t)gk * ldb + gj];
                    Bs[kk * 64 + c] = v;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    cx<R> a0 = As[kk * 64 + ty * 2], a1 = As[kk * 64 + ty * 2 + 1];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        cx<R> b = Bs[kk * 64 + tx * 4 + c];
                        acc[0][c] = cmac(acc[0][c], a0, b, false);
                        acc[1][c] = cmac(acc[1][c], a1, b, false);
                    }
                }
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                int gi = i0 + ty * 2 + r;
                if (gi >= m) continue;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    int gj = j0 + tx * 4 + c;
                    if (gj >= n) continue;
                    cx<R>* p = C + (size_t)gi * ldc + gj;
                    const cx<R> v = acc[r][c];
                    if (mode == GEMM_SET) *p = v;
                    else if (mode == GEMM_ADD) *p = cadd(*p, v);
                    else *p = csub(*p, v);
                }
            }
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Blocked Gauss-Jordan inverse with partial (row) pivoting.
//   A (K x K, leading dim lda, row-major on entry) is destroyed; A^-1 is written
//   to G (row-major, ldg).  The elimination runs on W = A^T, which the
//   row-major input already is when read column-major (W(i, l) = A[l*lda + i]):
//   the columns of W are contiguous, so every column-wise phase below reads
//   and writes contiguous memory.  The copy-out transposes back:
//   A^-1 = (W^-1)^T.
//   Pivots are taken in blocks of b columns.  For a block starting at j0 the
//   K x b panel W[:, j0:j0+b] is copied to shared memory and reduced there by
//   the unblocked in-place steps (pick the row p >= j with the largest
//   |W[p][j]|, swap rows j and p -- in the panel and in the rest of the matrix
//   --, scale the pivot row by 1/W[j][j] keeping 1/W[j][j] in column j,
//   eliminate column j from every other row keeping -W[i][j]/W[j][j] in
//   column j), recording for each step its multipliers c_jj[i] (column j at
//   row i just before step jj) and its pivot reciprocal.  The columns outside
//   the panel then receive the same b steps in two passes:
//     pivot rows (forward substitution, then the later steps' eliminations)
//       x_jj = (W[j0+jj][l] - sum_{jj' < jj} c_jj'[j0+jj] x_jj') / p_jj
//       W[j0+jj][l] = x_jj - sum_{jj' > jj} c_jj'[j0+jj] x_jj'
//     every other row (one rank-b update)
//       W[i][l] -= sum_jj c_jj[i] x_jj
//   (the second line for the pivot rows is the same update, started from x_jj
//   with the pivot rows' earlier multipliers set to zero, so one product
//   serves every row)
//   -- the arithmetic of the unblocked algorithm in a different association,
//   reading and writing each element once per block instead of once per pivot.
//   The substitution runs over all (pivot row, column) pairs of the block at
//   once -- the forward part right-looking, one block barrier per pivot, the
//   sums in the order above -- after the block's row swaps are applied to each
//   column as one permutation.  The row swaps are undone at the end by a
//   column permutation applied while copying into G.  Pivot reciprocals are
//   formed in the working precision (a Newton step on the binary32
//   reciprocal for double-float).  The pivot search is folded into the
//   previous pass: the threads that produce the next pivot column rank its
//   candidates by |a|^2 (binary32) and row index with a shared-memory atomic
//   maximum.  The pivot test runs in binary32 and falls back to binary64 near
//   its limits.
//   With a team of C blocks (one cluster) every block reduces the panel (the
//   same data, the same result) and updates only its own range of columns;
//   the copy-out is split by rows of G.  G is complete after the caller's next
//   cluster barrier.
// Returns a flag: bit 0 = zero pivot, or a pivot below 64 u sqrt(amax2) with
// amax2 = max |A_ij|^2 supplied by the caller (0 disables the test); bit 1 =
// non-finite pivot.
// ---------------------------------------------------------------------------
// Ranking key of a pivot candidate: |a|^2 in binary32 (NaN ranked as +inf)
// in the high word, the complement of the row in the low word -- the largest
// key is the largest magnitude and, among equal magnitudes, the lowest row.
template <class R>
__device__ __forceinline__ unsigned long long pivot_key(cx<R> v, int i) {
    float m = cabs2f(v);
    if (isnan(m)) m = INFINITY;
    return ((unsigned long long)__float_as_uint(m) << 32) | (0xFFFFFFFFu - (unsigned)i);
}

// Division by a divisor fixed for a loop: floor(n / d) = umulhi(n, ceil(2^32/d)),
// exact for n, d < 2^16 (the error n/2^32 stays below 1/d).
struct FastDiv {
    uint32_t d, m;
    __device__ explicit FastDiv(int dv) : d((uint32_t)dv), m(dv > 1 ? (uint32_t)((0x100000000ull + dv - 1) / dv) : 0u) {}
    __device__ int div(int n) const { return d == 1u ? n : (int)__umulhi((uint32_t)n, m); }
};

template <class R>
struct GJSmem {
    cx<R>* panel;    // [Kmax][bmax]  working panel
    cx<R>* panel2;   // [Kmax][bmax]  second panel buffer
    cx<R>* mult;     // [bmax][Kmax]  multipliers c_jj[i] at mult[jj*K + i]
    cx<R>* xrow;     // [bmax][Kmax]  substituted pivot rows outside the panel
    cx<R>* pinv;     // [bmax]   pivot reciprocals
    int* perm;       // [Kmax]
    int* idx;        // [Kmax]   row labels during the sweep, column order at the end
    int* pm;         // [2 bmax + 1]  rows displaced by a panel's swaps: count, rows, sources
    int* ctl;        // [4]: [1] = the pivot flags
    unsigned long long* key;   // [3]  pivot keys, one per pass, rotating
    int bmax;        // panel width
    tc::State* tcs;  // tensor-core state for the rank-b update, or nullptr
};

// The rank-b update of cta_gj_invert as a tensor-core product over one tile
// of up to 128 rows: W[i][l] -= sum_jj c_jj[i] x_jj[l] for the block's own
// columns l outside the panel (column c of the product -> l = col(c)) and
// every row i; a pivot row j0 + r starts from x_r instead of W.  The
// multipliers and pivot rows are read from shared memory (byte offsets into
// the dynamic shared memory); W is column-major, so the 32 rows a warp drains
// are contiguous.
struct GJUpdateOp {
    int cm_off;      // multipliers [bm][K]
    int xr_off;      // substituted pivot rows [bm][K]
    zf* A;
    int K, lda, r0, j0, bb, clo, ps, pskip;
    __device__ int col(int c) const { const int l = clo + c; return l < ps ? l : l + pskip; }
    __device__ zf a(int m, int k) const {
        return reinterpret_cast<const zf*>(rgf_dyn_smem + cm_off)[k * K + r0 + m];
    }
    __device__ zf b(int k, int n) const {
        return reinterpret_cast<const zf*>(rgf_dyn_smem + xr_off)[k * K + col(n)];
    }
    using Old = float4;
    __device__ bool colA() const { return true; }
    // the current value: W for other rows, x_r (shared memory) for the pivot rows
    __device__ float4 load(int m, int n, bool) const {
        const int i = r0 + m;
        if (i >= j0 && i < j0 + bb)
            return reinterpret_cast<const float4*>(rgf_dyn_smem + xr_off)[(i - j0) * K + col(n)];
        return *reinterpret_cast<const float4*>(A + (size_t)col(n) * lda + i);
    }
    __device__ void store(int m, int n, float4 x, df32 re, df32 im, bool) const {
        const df32 r = df_sub(df32{x.x, x.y}, re), q = df_sub(df32{x.z, x.w}, im);
        *reinterpret_cast<float4*>(A + (size_t)col(n) * lda + r0 + m) = make_float4(r.hi, r.lo, q.hi, q.lo);
    }
};

// The same rank-b update on binary64 data (RGF_FP64_TC): multipliers, pivot
// rows and W binary64, sliced from binary64, the update summed in binary64.
struct GJUpdateOp64 {
    static constexpr bool kF64 = true;
    int cm_off;      // multipliers [bm][K]
    int xr_off;      // substituted pivot rows [bm][K]
    zd* A;
    int K, lda, r0, j0, bb, clo, ps, pskip;
    __device__ int col(int c) const { const int l = clo + c; return l < ps ? l : l + pskip; }
    __device__ zd a(int m, int k) const {
        return reinterpret_cast<const zd*>(rgf_dyn_smem + cm_off)[k * K + r0 + m];
    }
    __device__ zd b(int k, int n) const {
        return reinterpret_cast<const zd*>(rgf_dyn_smem + xr_off)[k * K + col(n)];
    }
    using Old = zd;
    __device__ bool colA() const { return true; }
    __device__ zd load(int m, int n, bool) const {
        const int i = r0 + m;
        if (i >= j0 && i < j0 + bb) return reinterpret_cast<const zd*>(rgf_dyn_smem + xr_off)[(i - j0) * K + col(n)];
        return A[(size_t)col(n) * lda + i];
    }
    __device__ void store(int m, int n, zd x, double re, double im, bool) const {
        A[(size_t)col(n) * lda + r0 + m] = zd{x.re - re, x.im - im};
    }
};

// TC64: with R = double, run the rank-b updates on the tensor cores (binary64
// slicing) when the block holds them.
template <class R, bool TC64 = false>
__device__ int cta_gj_invert(cx<R>* __restrict__ A, int K, int lda, cx<R>* __restrict__ G, int ldg,
                             GJSmem<R> s, double amax2 = 0.0, Team tm = Team{0, 1}) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int bm = s.bmax;
    cx<R>* Pn = s.panel;
    cx<R>* Cm = s.mult;
    cx<R>* Xr = s.xrow;
    const double tiny2 = amax2 * (64.0 * Unit<R>::u) * (64.0 * Unit<R>::u);
    const int clo = tm.lo(K), chi = tm.hi(K);     // this block's columns of W
    const int rlo = tm.lo(K), rhi = tm.hi(K);     // this block's rows of G (copy-out)
    const float tiny2f = (float)tiny2;
    if (tid == 0) s.ctl[1] = 0;
    if (tid < 3) s.key[tid] = 0ull;
    for (int i = tid; i < K; i += NT) s.idx[i] = i;
    __syncthreads();
    for (int j0 = 0; j0 < K; j0 += bm) {
        const int bb = min(bm, K - j0);
        cx<R>* Pa = s.panel;            // panel, current
        cx<R>* Pb = s.panel2;           // panel, next
        unsigned long long kmax = 0ull;
        for (int e = tid; e < K * bb; e += NT) {
            const int i = e % K, jj = e / K;
            const cx<R> v = A[(size_t)(j0 + jj) * lda + i];
            Pa[i * bm + jj] = v;
            if (jj == 0 && i >= j0) kmax = max(kmax, pivot_key(v, i));
        }
        if (kmax) atomicMax(&s.key[j0 % 3], kmax);
        __syncthreads();
        for (int jj = 0; jj < bb; ++jj) {
            const int j = j0 + jj;
            // Every warp takes the pivot row from the key the previous pass
            // left and forms the reciprocal (lane 0, then broadcast), so no
            // barrier separates the pivot choice from the elimination; warp 0
            // records the pivot, the flags and the reciprocal.
            cx<R> invR = czero<R>();
            int p = 0;
            if (lane == 0) {
                const unsigned long long kj = s.key[j % 3];
                p = (int)(0xFFFFFFFFu - (unsigned)(kj & 0xFFFFFFFFull));
                cx<R> pv = Pa[p * bm + jj];
                int bad = 0;
                const float df = cabs2f(pv);
                if (!cfinite(pv)) {
                    bad = 2;
                } else if (!(df >= 1e-30f && df <= 1e30f && df >= 2.0f * tiny2f)) {
                    const double d = cabs2(pv);       // borderline: decide in binary64
                    if (!isfinite(d)) bad = 2;
                    else if (!(d > 0.0)) bad = 1;
                    else if (d < tiny2) bad = 1;
                }
                if (bad) pv = from_z<R>(1.0, 0.0);
                invR = crecip(pv);
                if (warp == 0) {
                    s.ctl[1] |= bad;
                    s.perm[j] = p;
                    s.pinv[jj] = invR;
                    s.key[(j + 2) % 3] = 0ull;   // read one pass ago, filled next pass
                }
            }
            invR = shfl0(invR);
            p = __shfl_sync(0xffffffffu, p, 0);
            // One pass: row swap j <-> p folded in as an index remap, pivot row
            // scaled, column jj eliminated from every other row (old -> new),
            // and the candidates for the next pivot ranked on the fly.
            // Threads: 16 columns x (NT / 16) rows, four rows per round (loads
            // first, then the arithmetic).
            const int l = tid & 15;
            kmax = 0ull;
            if (l < bb) {
                const cx<R> r = (l == jj) ? invR : cmul(Pa[p * bm + l], invR);
                constexpr int RS = NT / 16;
                for (int i0 = tid >> 4; i0 < K; i0 += 4 * RS) {
                    cx<R> mv[4], av[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + u * RS;
                        const int si = (i == j) ? p : ((i == p) ? j : i);
                        if (i < K && i != j) {
                            mv[u] = Pa[si * bm + jj];
                            av[u] = (l == jj) ? czero<R>() : Pa[si * bm + l];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int i = i0 + u * RS;
                        if (i >= K) continue;
                        if (i == j) {
                            Pb[i * bm + l] = r;
                        } else {
                            const cx<R> v = cmac(av[u], mv[u], r, true);
                            Pb[i * bm + l] = v;
                            if (l == jj) Cm[jj * K + i] = mv[u];
                            if (l == jj + 1 && i > j) kmax = max(kmax, pivot_key(v, i));
                        }
                    }
                }
            }
            kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, 16));
            if (lane == jj + 1 && kmax) atomicMax(&s.key[(j + 1) % 3], kmax);
            if (tid == 0) Cm[jj * K + j] = czero<R>();
            if (p != j)                  // earlier multipliers follow their rows
                for (int q = tid; q < jj; q += NT) {
                    cx<R> a = Cm[q * K + j];
                    Cm[q * K + j] = Cm[q * K + p];
                    Cm[q * K + p] = a;
                }
            __syncthreads();
            cx<R>* t = Pa; Pa = Pb; Pb = t;
        }
        // The block's row swaps as one permutation: idx[r] = the row whose
        // content row r holds after the swaps (identity outside the touched
        // rows); pm lists the displaced rows outside the panel and their sources.
        if (tid == 0) {
            int n = 0;
            for (int jj = 0; jj < bb; ++jj) {
                const int j = j0 + jj, p = s.perm[j];
                if (p != j) {
                    const int a = s.idx[j]; s.idx[j] = s.idx[p]; s.idx[p] = a;
                    if (p >= j0 + bb) s.pm[1 + n++] = p;
                }
            }
            for (int t = 0; t < n; ++t) s.pm[1 + bm + t] = s.idx[s.pm[1 + t]];
            s.pm[0] = n;
        }
        __syncthreads();
        // This block's columns outside the panel: the swaps, then the pivot
        // rows by block-wide substitution ...
        const int ps = max(j0, clo), pe = min(j0 + bb, chi);
        const int pskip = max(0, pe - ps);
        const int nown = (chi - clo) - pskip;            // own columns outside the panel
        auto own_col = [&](int c) { int l = clo + c; return (l < ps) ? l : l + pskip; };
        {
            // pivot rows after the swaps into Xr (x_0 scaled); tasks (r, c) with
            // r fastest so that a warp reads contiguous rows of one column
            const FastDiv dbb(bb), down(max(nown, 1));
            for (int e = tid; e < bb * nown; e += NT) {
                const int c = dbb.div(e), r = e - c * bb, l = own_col(c);
                cx<R> v = A[(size_t)l * lda + s.idx[j0 + r]];
                if (r == 0) v = cmul(v, s.pinv[0]);
                Xr[r * K + l] = v;
            }
            __syncthreads();
            // rows outside the panel that took a panel row's content (the
            // sources are panel rows, unchanged until the stores below)
            const int npm = s.pm[0];
            const FastDiv dpm(max(npm, 1));
            for (int e = tid; e < npm * nown; e += NT) {
                const int c = dpm.div(e), t = e - c * npm;
                cx<R>* colp = A + (size_t)own_col(c) * lda;
                colp[s.pm[1 + t]] = colp[s.pm[1 + bm + t]];
            }
            // forward substitution, right-looking: after step q every later
            // pivot row has subtracted c_q x_q (the sums keep their order), and
            // row q + 1 is final and scaled
            for (int q = 0; q + 1 < bb; ++q) {
                const int nr = bb - 1 - q;
                for (int e = tid; e < nr * nown; e += NT) {
                    const int rr = down.div(e), c = e - rr * nown, r = q + 1 + rr, l = own_col(c);
                    cx<R> a = cmac(Xr[r * K + l], Cm[q * K + j0 + r], Xr[q * K + l], true);
                    if (r == q + 1) a = cmul(a, s.pinv[r]);
                    Xr[r * K + l] = a;
                }
                __syncthreads();
            }
            // The later steps' eliminations of the pivot rows,
            //   W[j0+r][l] = x_r - sum_{q > r} c_q[j0+r] x_q,
            // have the form of the rank-b update below; with the pivot rows'
            // multipliers of the earlier steps (q <= r) set to zero the update
            // produces them from x_r.
            for (int e = tid; e < bb * bb; e += NT) {
                const int r = e / bb, q = e % bb;
                if (q < r) Cm[q * K + j0 + r] = czero<R>();
            }
        }
        __syncthreads();
        if (tid == 0) {                  // labels back to the identity
            for (int jj = 0; jj < bb; ++jj) s.idx[j0 + jj] = j0 + jj;
            for (int t = 0; t < s.pm[0]; ++t) s.idx[s.pm[1 + t]] = s.pm[1 + t];
        }
        Pn = Pa;                         // the reduced panel
        // ... then one rank-bb update of every row (the pivot rows from x_r):
        // on the tensor cores (double-float operands, exact digit slicing) or
        // on the FP32 / FP64 pipes.
        bool tc_done = false;
        if constexpr (std::is_same<R, df32>::value) {
            if (s.tcs && nown > 0) {
                const int cm_off = tc::dyn_off(Cm), xr_off = tc::dyn_off(Xr);
                for (int r0 = 0; r0 < K; r0 += 128) {
                    const GJUpdateOp op{cm_off, xr_off, A, K, lda, r0, j0, bb, clo, ps, pskip};
                    s.tcs->phase = tc::zgemm(op, min(128, K - r0), nown, bb, s.tcs->ar, s.tcs->phase);
                }
                tc_done = true;
            }
        } else if constexpr (std::is_same<R, double>::value && TC64) {
            if (s.tcs && nown > 0) {
                const int cm_off = tc::dyn_off(Cm), xr_off = tc::dyn_off(Xr);
                for (int r0 = 0; r0 < K; r0 += 128) {
                    const GJUpdateOp64 op{cm_off, xr_off, A, K, lda, r0, j0, bb, clo, ps, pskip};
                    s.tcs->phase = tc::zgemm(op, min(128, K - r0), nown, bb, s.tcs->ar, s.tcs->phase);
                }
                tc_done = true;
            }
        }
        const int Kh = (K + 1) >> 1, Ch = tc_done ? 0 : (nown + 1) >> 1;
        for (int tt = tid; tt < Kh * Ch; tt += NT) {
            const int i0 = 2 * (tt % Kh), c0 = 2 * (tt / Kh);
            const bool ok_i1 = i0 + 1 < K, ok_c1 = c0 + 1 < nown;
            const int l0 = own_col(c0);
            const int l1 = ok_c1 ? own_col(c0 + 1) : l0;
            // the current value: W for other rows, x_r for the pivot rows
            auto cur = [&](int i, int l) {
                return (i >= j0 && i < j0 + bb) ? Xr[(i - j0) * K + l] : A[(size_t)l * lda + i];
            };
            cx<R> a00 = cur(i0, l0), a01 = czero<R>(), a10 = czero<R>(), a11 = czero<R>();
            if (ok_c1) a01 = cur(i0, l1);
            if (ok_i1) {
                a10 = cur(i0 + 1, l0);
                if (ok_c1) a11 = cur(i0 + 1, l1);
            }
            for (int jj = 0; jj < bb; ++jj) {
                const cx<R> p0 = Cm[jj * K + i0];
                const cx<R> p1 = ok_i1 ? Cm[jj * K + i0 + 1] : czero<R>();
                const cx<R> m0 = Xr[jj * K + l0];
                const cx<R> m1 = ok_c1 ? Xr[jj * K + l1] : czero<R>();
                a00 = cmac(a00, p0, m0, true);
                a01 = cmac(a01, p0, m1, true);
                a10 = cmac(a10, p1, m0, true);
                a11 = cmac(a11, p1, m1, true);
            }
            cx<R>* c0p = A + (size_t)l0 * lda;
            cx<R>* c1p = A + (size_t)l1 * lda;
            c0p[i0] = a00;
            if (ok_c1) c1p[i0] = a01;
            if (ok_i1) {
                c0p[i0 + 1] = a10;
                if (ok_c1) c1p[i0 + 1] = a11;
            }
        }
        // the reduced panel: this block's part of its rows
        for (int e = tid; e < (rhi - rlo) * bb; e += NT) {
            const int i = rlo + e % (rhi - rlo), jj = e / (rhi - rlo);
            A[(size_t)(j0 + jj) * lda + i] = Pn[i * bm + jj];
        }
        cl_sync(tm);
    }
    if (tid == 0) {
        for (int c = 0; c < K; ++c) s.idx[c] = c;
        for (int j = K - 1; j >= 0; --j) {
            int p = s.perm[j];
            int tmp = s.idx[j]; s.idx[j] = s.idx[p]; s.idx[p] = tmp;
        }
    }
    __syncthreads();
    // G = (W^-1)^T with the row swaps undone: G[i][c] = W[c][idx[i]]
    for (int i = rlo + warp; i < rhi; i += NWARP) {
        const cx<R>* col = A + (size_t)s.idx[i] * lda;
        cx<R>* grow = G + (size_t)i * ldg;
        for (int c = lane; c < K; c += 32) grow[c] = col[c];
    }
    const int flag = s.ctl[1];
    __syncthreads();
    return flag;
}

}  // namespace rgf
