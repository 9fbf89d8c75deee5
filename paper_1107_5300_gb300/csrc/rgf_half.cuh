// rgf_half.cuh -- the RGF recursion (Eqs. 4-5) and the Landauer trace (Eq. 2)
// for a batch of chains (ribbon, energy), as two half sweeps per chain joined
// by one Dyson step (Eq. 3).
//
// The paper slices the ribbon into cross-sections and applies, slice after
// slice, g_j = (z - H_jj - V^T g_{j-1} V)^-1 together with the corner block
// G_1j = G_1,j-1 V g_j (Eqs. 4-5).  Here each unit cell (2N orbitals) is
// sliced further into its four atom columns (x = 0, a, 1.5a, 2.5a): a column
// has no internal hopping, neighbouring columns are coupled by t*I (same row)
// or by a bidiagonal t-stencil (rows j +- 1).  The recursion is the same
// Dyson step on blocks of KL = ceil(N/2) or KR = floor(N/2) orbitals, 4L
// columns per chain.
//
// Domain decomposition.  A chain's recursion is strictly sequential along the
// ribbon; the paper notes that running it in parallel needs a modified
// recursion (its remark on MPI).  The columns 0 .. n-1 (n = 4L) are cut into
// a left part 0 .. m-1 and a right part m .. n-1 (m = n/2).  Each part runs
// the recursion from its own lead, on its own SM, at the same time:
//
//   left  (k = 0 .. m-1):   gl_k = (z - eps_k - t^2 S_k^T gl_{k-1} S_k)^-1
//                           Pl_k = U_even^T G^left_{0,k}  = Pl_{k-1} W_k gl_k
//   right (k = n-1 .. m):   gr_k = (z - eps_k - t^2 S_{k+1} gr_{k+1} S_{k+1}^T)^-1
//                           Pr_k = U_odd^T G^right_{n-1,k} = Pr_{k+1} W_{k+1}^T gr_k
//
// (W_k = t S_k the coupling of columns k-1 and k; each part sees only its own
// lead.)  The Dyson equation across the bond between columns m-1 and m then
// gives the corner block of the whole system,
//
//   G_{0,n-1} = G^left_{0,m-1} W_m (I - gr_m SigmaL_m)^-1 G^right_{m,n-1},
//   SigmaL_m = W_m^T gl_{m-1} W_m,
//
// so U_even^T G_{0,n-1} U_odd = (Pl_{m-1} W_m) (I - gr_m SigmaL_m)^-1 Pr_m^T and
// T = sum_pq gamma_p gamma'_q |(U_even^T G_{0,n-1} U_odd)_pq|^2 (Eq. 2 in the
// mode basis, gamma = -2 Im w).  Same work as one sweep over n columns, half
// the sequential depth.
//
// Lead-attached columns.  The first column of each part carries the lead
// self-energy, Sigma = U diag(w) U^T.  Near E = 0 the transverse cut of an
// armchair ribbon is zigzag-like and the modes with |tau_p| > |t| have a
// surface state: |w_p| ~ 1/eta (~1e9 eV at eta = 1e-8).  In the site basis
// those entries would be summed with the order-1 on-site terms and drown
// them.  The first column is therefore formed and inverted in the mode basis,
// in binary64, by its own kernel (prep_kernel):
//
//   A~ = U^T diag(z - eps) U - diag(w),   g~ = A~^-1,
//   P_0 = g~ U^T (rows in the mode basis),   g_0 = U P_0 (site basis),
//
// where the surface-state modes meet only their own order-1/eta diagonal.
// The corner blocks are carried with their rows in the mode bases, so the
// order-eta components that Gamma ~ 1/eta weights in the trace keep their own
// relative accuracy.  (A lead-attached column with a removed atom is formed
// in the site basis instead.)
//
// Two schedules share the device bodies below (prep_body, half_body,
// merge_body): three launches per call (rgf_sweep.cu: prep_kernel, binary64, 2
// blocks per chain; half_kernel<R, TC>, the recursion of each part, 2 blocks
// per chain, the dominant kernel; merge_kernel, binary64, 1 block per chain:
// the Dyson step across the cut, the trace and the status word), or one
// persistent kernel with a work queue (rgf_batch.cu).  Removed atoms become
// identity rows/columns with zero couplings (an exact equivalence to dropping
// them).  With TC (RGF_MIXED_TC, RGF_FP64_TC) the two dense contractions of a
// column step -- the Gauss-Jordan rank-b updates and the strip product -- run
// on the tcgen05 tensor cores by exact digit slicing of their operands
// (rgf_tc.cuh); every block then holds the SM's TMEM for the launch.
#pragma once

#include "rgf_steps.cuh"

namespace rgf {
namespace {

// Columns of the left part; the right part has ncol - m.
__host__ __device__ inline int left_cols(int ncol) { return ncol / 2; }

// The buffers of one half of a chain's workspace (16-byte elements, ld KL).
template <class R>
struct Half {
    cx<R>* X;        // slice matrix / scratch
    cx<R>* G;        // g of the last column done
    cx<R>* P;        // corner block, rows in the lead's mode basis
    int* flag;       // Gauss-Jordan / tensor-core flags of this half
};
template <class R>
__device__ inline Half<R> half_of(void* ws, const ChainDev& ch, int h) {
    const size_t B = (size_t)col_KL(ch.N) * col_KL(ch.N);
    cx<R>* base = reinterpret_cast<cx<R>*>(ws) + ch.ws_off + (size_t)h * half_ws_elems(ch.N);
    return Half<R>{base, base + B, base + 2 * B, reinterpret_cast<int*>(base + 3 * B)};
}

// In-place conversion of a K1 x K2 block (ld) between binary64 and the
// working precision (both 16-byte complex elements).  Every thread; barrier.
template <class R>
__device__ void to_working(cx<R>* p, int K1, int K2, int ld) {
    for (int e = threadIdx.x; e < K1 * K2; e += NT) {
        const int i = e / K2, j = e % K2;
        const zd v = reinterpret_cast<zd*>(p)[(size_t)i * ld + j];
        p[(size_t)i * ld + j] = from_z<R>(v.re, v.im);
    }
    __syncthreads();
}
template <class R>
__device__ void to_binary64(cx<R>* p, int K1, int K2, int ld) {
    for (int e = threadIdx.x; e < K1 * K2; e += NT) {
        const int i = e / K2, j = e % K2;
        const zd v = to_z(p[(size_t)i * ld + j]);
        reinterpret_cast<zd*>(p)[(size_t)i * ld + j] = v;
    }
    __syncthreads();
}

__device__ inline double max_abs2(const zd* A, int K, int ld, double* red) {
    double m = 0.0;
    for (int e = threadIdx.x; e < K * K; e += NT) {
        const double a = cabs2(A[(size_t)(e / K) * ld + e % K]);
        m = (a > m || isnan(a)) ? a : m;
    }
    return block_max(m, red);
}

// Everything the sweep kernels read besides their own shared memory.
struct SweepArgs {
    const ChainDev* chains;
    const int* order;
    int nchains, Kmax;
    double eta_d;
    const zd* leadout;
    const int* lead_status;
    const LeadDev* leads;
    void* ws;
    double* T;
    int32_t* status;
    int ndom;        // domains per chain (2: the two halves)
};

// The buffers of interior domain d (1 .. ndom-2) of a chain (ld KL): for its
// columns a .. b, the left-connected recursion of the isolated domain leaves
// G = g_b, P = G_ab (rows: column a) and A = G_aa.
template <class R>
struct Inner {
    cx<R>* X;
    cx<R>* G;
    cx<R>* P;
    cx<R>* A;
    int* flag;
};
template <class R>
__device__ inline Inner<R> inner_of(void* ws, const ChainDev& ch, int d) {
    const size_t B = (size_t)col_KL(ch.N) * col_KL(ch.N);
    cx<R>* base = reinterpret_cast<cx<R>*>(ws) + ch.ws_off + sweep_ws_elems(ch.N) +
                  (size_t)(d - 1) * interior_ws_elems(ch.N);
    return Inner<R>{base, base + B, base + 2 * B, base + 3 * B, reinterpret_cast<int*>(base + 4 * B)};
}

// The lead-attached first column of half h of chain ci, in binary64: h = 0 the
// left lead's column 0 (KL even-row left atoms), h = 1 the right lead's column
// n-1 (KR odd-row right atoms).  Writes g (site basis) and P (rows in the
// lead's mode basis) into the half's G and P in the working precision R, and
// the Gauss-Jordan flags into the half's flag word.  bm: the launch's panel
// width.  Every thread; ends with a barrier.
template <class R>
__device__ __noinline__ void prep_body(const SweepArgs a, int ci, int h, int bm) {
    SweepSmem<double> s = carve<double>(rgf_dyn_smem, a.Kmax, false, bm);
    const ChainDev& ch = a.chains[ci];
    const ChainCtx c = make_ctx(ch, a.leads[ch.lead], a.leadout, a.eta_d, h);
    const Half<R> hw = half_of<R>(a.ws, ch, h);
    zd* X = reinterpret_cast<zd*>(hw.X);
    zd* G = reinterpret_cast<zd*>(hw.G);
    zd* P = reinterpret_cast<zd*>(hw.P);
    const int KL = c.KL, k = h ? c.ncol - 1 : 0, K = h ? c.KR : c.KL;
    const zd* U = h ? c.UR() : c.UL();                  // K x K, ld K
    const zd* Sig = h ? c.SigR() : c.SigL();            // K x K, ld K
    load_col(c, k, s.kc, s.eps);
    if (threadIdx.x == 0) s.gj.ctl[2] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < K; i += NT)
        if (!s.kc[i]) s.gj.ctl[2] = 1;
    __syncthreads();
    const bool removed = s.gj.ctl[2] != 0;
    int flag;
    if (!removed) {
        // A~ = U^T diag(z - eps) U - diag(w) into G; g~ = A~^-1 into X
        for (int e = threadIdx.x; e < K * K; e += NT) {
            const int i = e / K, p = e % K;
            const double u = U[(size_t)i * K + p].re;
            X[(size_t)i * KL + p] = {(c.z.re - s.eps[i]) * u, c.z.im * u};
        }
        __syncthreads();
        cta_gemm<double, true, false>(K, K, K, U, K, X, KL, G, KL, GEMM_SET, s.gemm);
        for (int p = threadIdx.x; p < K; p += NT) G[(size_t)p * KL + p] = csub(G[(size_t)p * KL + p], c.w()[p]);
        __syncthreads();
        const double amax2 = max_abs2(G, K, KL, s.red);
        flag = cta_gj_invert<double>(G, K, KL, X, KL, s.gj, amax2);
        // P = g~ U^T, then g = U P
        cta_gemm<double, false, true>(K, K, K, X, KL, U, K, P, KL, GEMM_SET, s.gemm);
        cta_gemm<double, false, false>(K, K, K, U, K, P, KL, G, KL, GEMM_SET, s.gemm);
    } else {
        // site basis: (z - eps) I - Sigma on the kept atoms, identity rows and
        // columns at removed atoms; then P = U^T g
        for (int e = threadIdx.x; e < K * K; e += NT) {
            const int i = e / K, l = e % K;
            zd v;
            if (!s.kc[i] || !s.kc[l]) v = (i == l) ? zd{1.0, 0.0} : zd{0.0, 0.0};
            else v = csub((i == l) ? zd{c.z.re - s.eps[i], c.z.im} : zd{0.0, 0.0}, Sig[(size_t)i * K + l]);
            X[(size_t)i * KL + l] = v;
        }
        __syncthreads();
        const double amax2 = max_abs2(X, K, KL, s.red);
        flag = cta_gj_invert<double>(X, K, KL, G, KL, s.gj, amax2);
        cta_gemm<double, true, false>(K, K, K, U, K, G, KL, P, KL, GEMM_SET, s.gemm);
    }
    to_working<R>(hw.G, K, K, KL);
    to_working<R>(hw.P, K, K, KL);
    if (threadIdx.x == 0) *hw.flag = flag;
    __syncthreads();
}

// The recursion of half h of chain ci from its second column to the cut:
// columns 1 .. m-1 (left) or n-2 .. m (right), in pairs of t I-bonded columns
// wherever the chain's schedule and pair_ok allow (pair_column in
// rgf_steps.cuh), else one column at a time.  bm: the launch's panel width
// (the chain's schedule may narrow it); tst: the block's tensor-core state
// (TC).  ORs the Gauss-Jordan
// and tensor-core flags into the half's flag word.  Every thread; ends with a
// barrier.
template <class R, bool TC>
__device__ __forceinline__ void half_body(const SweepArgs& a, int ci, int h, int bm, tc::State* tst) {
    SweepSmem<R> s = carve<R>(rgf_dyn_smem, a.Kmax, TC, bm);
    const ChainDev& ch = a.chains[ci];
    const ChainCtx c = make_ctx(ch, a.leads[ch.lead], a.leadout, a.eta_d, h);
    const Half<R> hw = half_of<R>(a.ws, ch, h);
    const int m = left_cols(c.ncol), steps = h ? c.ncol - m : m;
    if (ch.panel > 0 && ch.panel < bm) s.gj.bmax = ch.panel;
    const bool pairs_on = ch.pairs != 0;
    if constexpr (TC) {
        s.gj.tcs = tst;
        s.tcs = tst;
    }
    int flag = 0;
    for (int j = 1; j < steps;) {
        const int k = h ? c.ncol - 1 - j : j;
        // a pair: this column and the next one in the recursion share t I bonds
        // (c0-c1 or c2-c3 of one cell); the second column of the first pair of
        // each half is the one after the prepared end column
        const int kb = h ? k - 1 : k + 1;
        const bool pairable = pairs_on && j + 1 < steps && (h ? (k & 1) == 1 : (k & 1) == 0);
        load_col(c, k, s.kc, s.eps);
        load_col(c, prev_col(c, k), s.kp, nullptr);
        if (pairable) load_col(c, kb, s.kn, nullptr);
        __syncthreads();
        const bool pair = pairable && pair_ok<R>(c, kb, s);
        // one call site each for the inverse and the strip product (inlined)
        flag |= inv_column<R, TC>(c, k, hw.G, hw.G, hw.X, s, pair ? kb : -1);
        if (pair) pair_scales<R>(c, k, kb, hw.G, s);
        strip_column<R, TC>(c, k, hw.G, hw.P, hw.P, hw.X, s);
        if (pair) pair_finish<R>(c, k, hw.G, s);
        j += pair ? 2 : 1;
    }
    if constexpr (TC) {
        if (*(volatile int*)tst->ar.err()) flag |= 4;
    }
    __syncthreads();
    if (threadIdx.x == 0) *hw.flag |= flag;
    __syncthreads();
}

// Domain d of chain ci when the chain has ndom > 2 domains, in one body for
// the three kinds (one inlined copy each of the inverse and the strip
// product):
//   d = 0, ndom-1: the lead-attached halves, as half_body (their end columns
//     prepared by prep_body), the left one ending before the first interior
//     domain, the right one starting at the last;
//   interior d: columns a = dom_bound(d) .. b = dom_bound(d + 1) - 1 as an
//     isolated system, recursed left to right.  It starts with its first two
//     columns, t I-bonded row by row: each row is a dimer [[d1, -t], [-t, d2]]
//     (d = z - eps), so A = G_aa = diag(d2 / D), P = G_a,a+1 = diag(t / D) and
//     G = g_a+1 = diag(d1 / D) with D = d1 d2 - t^2 (a removed atom leaves its
//     partner alone: 1 / d).  Column a also carries an absorbing self-energy
//     -i |t| on its kept atoms (d1 = z - eps + i |t|), which the join takes
//     back out exactly: an isolated segment has a discrete spectrum, and an
//     energy next to one of its levels would make its blocks, and the joins,
//     ill-conditioned; open at one end, like the halves, it is not.  Starting
//     from the dimers also keeps an atom near resonance (|z - eps| small) from
//     entering as an isolated 1 / (z - eps).  Each step then adds column k (or
//     a pair k, kb) to the partial system a .. k-1 by the Dyson equation:
//         g_k = (A_k - W_k^T g_{k-1} W_k)^-1                       (inv_column)
//         Y = P W_k,  P <- Y g_k,  A <- A + Y g_k Y^T = A + P Y^T  (G_aa, G_ab)
//     On return G = g_b, P = G_ab and A = G_aa of the isolated domain; the
//     joins in merge_body use them.
// A pair takes Z, the inverse of its shifted first column (the pair's own
// block at k): the strip forms (Y Z), the interior adds (Y Z) Y^T to A, and
// then P = (Y Z) diag(s) and g_kb = diag(1/d) + diag(s) Z diag(s)
// (pair_scales, pair_finish).  Every thread; ends with a barrier.
template <class R, bool TC>
__device__ __forceinline__ void domain_body(const SweepArgs& a, int ci, int d, int bm,
                                            tc::State* tst) {
    SweepSmem<R> s = carve<R>(rgf_dyn_smem, a.Kmax, TC, bm);
    const ChainDev& ch = a.chains[ci];
    const bool right = d == a.ndom - 1, inner = d > 0 && !right;
    const ChainCtx c = make_ctx(ch, a.leads[ch.lead], a.leadout, a.eta_d, right ? 1 : 0);
    const int KL = c.KL;
    cx<R> *X, *G, *P, *A = nullptr;
    int* fl;
    int k0, k1, rows;                   // columns k0 .. k1-1 (right half: k1-1 down to k0)
    if (inner) {
        const Inner<R> iw = inner_of<R>(a.ws, ch, d);
        X = iw.X; G = iw.G; P = iw.P; A = iw.A; fl = iw.flag;
        k0 = dom_bound(c.ncol, d, a.ndom);
        k1 = dom_bound(c.ncol, d + 1, a.ndom);
        rows = col_size(c, k0);
    } else {
        const Half<R> hw = half_of<R>(a.ws, ch, right ? 1 : 0);
        X = hw.X; G = hw.G; P = hw.P; fl = hw.flag;
        k0 = right ? dom_bound(c.ncol, a.ndom - 1, a.ndom) : 0;
        k1 = right ? c.ncol : dom_bound(c.ncol, 1, a.ndom);
        rows = right ? c.KR : c.KL;
    }
    if (ch.panel > 0 && ch.panel < bm) s.gj.bmax = ch.panel;
    const bool pairs_on = ch.pairs != 0;
    if constexpr (TC) {
        s.gj.tcs = tst;
        s.tcs = tst;
    }
    if (inner) {
        // the dimers of columns k0, k0 + 1 (binary64; same row, same size)
        const int K0 = rows;
        load_col(c, k0, s.kc, s.eps);
        load_col(c, k0 + 1, s.kn, nullptr);
        __syncthreads();
        for (int e = threadIdx.x; e < K0 * K0; e += NT) {
            const int i = e / K0, l = e - i * K0;
            zd ga = {0.0, 0.0}, gab = {0.0, 0.0}, gb = {0.0, 0.0};
            if (i == l) {
                const zd d1 = {c.z.re - s.eps[i], c.z.im + fabs(c.t)};
                const zd d2 = {c.z.re - site_eps(c, k0 + 1, i), c.z.im};
                const bool k1a = s.kc[i], k2a = s.kn[i];
                if (k1a && k2a) {
                    const zd det = csub(cmul(d1, d2), zd{c.t2, 0.0});
                    const zd r = crecip(det);
                    ga = cmul(d2, r);
                    gab = cscale(r, c.t);
                    gb = cmul(d1, r);
                } else {
                    ga = k1a ? crecip(d1) : zd{1.0, 0.0};
                    gb = k2a ? crecip(d2) : zd{1.0, 0.0};
                }
            }
            A[(size_t)i * KL + l] = from_z<R>(ga.re, ga.im);
            P[(size_t)i * KL + l] = from_z<R>(gab.re, gab.im);
            G[(size_t)i * KL + l] = from_z<R>(gb.re, gb.im);
        }
        __syncthreads();
    }
    const int steps = k1 - k0;
    int flag = 0;
    for (int j = inner ? 2 : 1; j < steps;) {
        const int k = right ? k1 - 1 - j : k0 + j;
        const int kb = right ? k - 1 : k + 1;
        const bool pairable = pairs_on && j + 1 < steps && (right ? (k & 1) == 1 : (k & 1) == 0);
        load_col(c, k, s.kc, s.eps);
        load_col(c, prev_col(c, k), s.kp, nullptr);
        if (pairable) load_col(c, kb, s.kn, nullptr);
        __syncthreads();
        const bool pair = pairable && pair_ok<R>(c, kb, s);
        const int K = col_size(c, k);
        flag |= inv_column<R, TC>(c, k, G, G, X, s, pair ? kb : -1);
        strip_column<R, TC>(c, k, G, P, P, X, s, rows);          // Y = P W into X, P <- Y G
        if (inner) acc_product<R, TC>(rows, K, P, X, A, KL, s);  // A += P Y^T
        if (pair) {
            pair_scales<R>(c, k, kb, G, s);                      // G = Z diag(s)
            const cx<R>* sc = s.gj.mult;
            for (int e = threadIdx.x; e < rows * K; e += NT) {
                const int i = e / K, l = e - i * K;
                P[(size_t)i * KL + l] = cmul(P[(size_t)i * KL + l], sc[l]);
            }
            __syncthreads();
            pair_finish<R>(c, k, G, s);
        }
        j += pair ? 2 : 1;
    }
    if constexpr (TC) {
        if (*(volatile int*)tst->ar.err()) flag |= 4;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (inner) *fl = flag;
        else *fl |= flag;
    }
    __syncthreads();
}

// One join of the tree that combines the interior domains (ndom > 3):
// at level l, join j combines node d1 = 1 + j 2^(l+1) (its domains d1 ..
// d1 + 2^l - 1) with node d2 = d1 + 2^l (domains d2 .. min(d2 + 2^l, ndom-1)
// - 1), both interior segments open only at their first column (the
// absorbing term -i|t|).  With a1 .. b1 and a2 .. b2 their columns, blocks
// A = G_aa, B = G_ab, D = g_b, and Sigma = W^T D1 W + i|t| on column a2 (the
// coupling from node 1 in place of node 2's absorbing term), the Dyson
// equation across the bond b1 -> a2 gives the combined segment a1 .. b2:
//     Y = (I - A2 Sigma)^-1 B2,             G'_a2a2 = (I - A2 Sigma)^-1 A2,
//     D' = D2 + B2^T Sigma Y,               B' = (B1 W) Y,
//     A' = A1 + (B1 W) G'_a2a2 (B1 W)^T,
// written into node d1's buffers in binary64 (level 0 converts its inputs
// from the working precision).  One inverse and seven products; a block per
// join, every join of a level at the same time.  TCJ (the tensor-core
// precisions): the products and the inverse's rank-b updates on the tensor
// cores, sliced from binary64 and summed in binary64 (the block holds TMEM,
// tst); else on the FP64 pipes.
template <class R, bool TCJ>
__device__ __noinline__ void tree_join_body(const SweepArgs a, int ci, int level, int j, int bm,
                                            tc::State* tst) {
    SweepSmem<double> s = carve<double>(rgf_dyn_smem, a.Kmax, TCJ, bm);
    if constexpr (TCJ) {
        s.gj.tcs = tst;
        s.tcs = tst;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const ChainDev& ch = a.chains[ci];
    const ChainCtx c = make_ctx(ch, a.leads[ch.lead], a.leadout, a.eta_d, 0);
    const int M = a.ndom - 2, w = 1 << level;
    const int d1 = 1 + j * 2 * w, d2 = d1 + w;
    const int KL = c.KL;
    if (d2 > M) {
        // an odd domain out at level 0 still goes over to binary64, as the
        // levels above expect
        if (level == 0 && d1 <= M) {
            const Inner<R> I = inner_of<R>(a.ws, ch, d1);
            const int ka = dom_bound(c.ncol, d1, a.ndom), kb = dom_bound(c.ncol, d1 + 1, a.ndom) - 1;
            to_binary64<R>(I.A, col_size(c, ka), col_size(c, ka), KL);
            to_binary64<R>(I.P, col_size(c, ka), col_size(c, kb), KL);
            to_binary64<R>(I.G, col_size(c, kb), col_size(c, kb), KL);
        }
        return;
    }
    const double t = c.t, t2 = c.t2;
    const int a1 = dom_bound(c.ncol, d1, a.ndom), b1 = dom_bound(c.ncol, d2, a.ndom) - 1;
    const int a2 = dom_bound(c.ncol, d2, a.ndom);
    const int b2 = dom_bound(c.ncol, min(d2 + w, a.ndom - 1), a.ndom) - 1;
    const int K1 = col_size(c, a1), Kb1 = col_size(c, b1), K2 = col_size(c, a2), Kb2 = col_size(c, b2);
    const Inner<R> I1 = inner_of<R>(a.ws, ch, d1), I2 = inner_of<R>(a.ws, ch, d2);
    if (level == 0) {
        to_binary64<R>(I1.A, K1, K1, KL);
        to_binary64<R>(I1.P, K1, Kb1, KL);
        to_binary64<R>(I1.G, Kb1, Kb1, KL);
        to_binary64<R>(I2.A, K2, K2, KL);
        to_binary64<R>(I2.P, K2, Kb2, KL);
        to_binary64<R>(I2.G, Kb2, Kb2, KL);
    }
    zd* X1 = reinterpret_cast<zd*>(I1.X);
    zd* A1 = reinterpret_cast<zd*>(I1.A);
    zd* B1 = reinterpret_cast<zd*>(I1.P);
    zd* D1 = reinterpret_cast<zd*>(I1.G);
    zd* X2 = reinterpret_cast<zd*>(I2.X);
    zd* A2 = reinterpret_cast<zd*>(I2.A);
    zd* B2 = reinterpret_cast<zd*>(I2.P);
    zd* D2 = reinterpret_cast<zd*>(I2.G);
    int flag = *I1.flag | *I2.flag;
    const int ct = a2 & 3;
    load_col(c, a2, s.kc, nullptr);
    load_col(c, b1, s.kp, nullptr);
    __syncthreads();
    // Sigma = t^2 S^T D1 S + i|t| on column a2 (kept atoms only) into X1
    for (int i = warp; i < K2; i += NWARP) {
        int p0, p1;
        col_src(ct, i, Kb1, p0, p1);
        const bool ki = s.kc[i];
        const bool kp0 = p0 >= 0 && s.kp[p0], kp1 = p1 >= 0 && s.kp[p1];
        for (int l = lane; l < K2; l += 32) {
            zd v = {0.0, 0.0};
            if (ki && s.kc[l]) {
                int q0, q1;
                col_src(ct, l, Kb1, q0, q1);
                const bool kq0 = q0 >= 0 && s.kp[q0], kq1 = q1 >= 0 && s.kp[q1];
                if (kp0 && kq0) v = cadd(v, D1[(size_t)p0 * KL + q0]);
                if (kp0 && kq1) v = cadd(v, D1[(size_t)p0 * KL + q1]);
                if (kp1 && kq0) v = cadd(v, D1[(size_t)p1 * KL + q0]);
                if (kp1 && kq1) v = cadd(v, D1[(size_t)p1 * KL + q1]);
                v = cscale(v, t2);
                if (i == l) v.im += fabs(t);
            }
            X1[(size_t)i * KL + l] = v;
        }
    }
    __syncthreads();
    // X = I - A2 Sigma into X2; B2^T Sigma into D1 (D1 read for the last time)
    dense_product<double, false, TCJ>(K2, K2, K2, A2, KL, X1, KL, X2, KL, s);
    for (int e = threadIdx.x; e < K2 * K2; e += NT) {
        const int i = e / K2, l = e % K2;
        zd& x = X2[(size_t)i * KL + l];
        x = {((i == l) ? 1.0 : 0.0) - x.re, -x.im};
    }
    __syncthreads();
    dense_product<double, true, TCJ>(Kb2, K2, K2, B2, KL, X1, KL, D1, KL, s);
    // X^-1 into X1; Y = X^-1 B2 into X2; G'_a2a2 = X^-1 A2 into B2
    const double amax2 = max_abs2(X2, K2, KL, s.red);
    flag |= cta_gj_invert<double, TCJ>(X2, K2, KL, X1, KL, s.gj, amax2);
    dense_product<double, false, TCJ>(K2, Kb2, K2, X1, KL, B2, KL, X2, KL, s);
    dense_product<double, false, TCJ>(K2, K2, K2, X1, KL, A2, KL, B2, KL, s);
    // D' = D2 + (B2^T Sigma) Y into A2, then into D1's place below
    dense_product<double, false, TCJ>(Kb2, Kb2, K2, D1, KL, X2, KL, A2, KL, s);
    for (int e = threadIdx.x; e < Kb2 * Kb2; e += NT) {
        const int i = e / Kb2, l = e % Kb2;
        A2[(size_t)i * KL + l] = cadd(A2[(size_t)i * KL + l], D2[(size_t)i * KL + l]);
    }
    // B1 W (K1 x K2) into X1
    for (int r = warp; r < K1; r += NWARP)
        for (int l = lane; l < K2; l += 32) {
            zd v = {0.0, 0.0};
            if (s.kc[l]) {
                int p0, p1;
                col_src(ct, l, Kb1, p0, p1);
                if (p0 >= 0 && s.kp[p0]) v = cadd(v, B1[(size_t)r * KL + p0]);
                if (p1 >= 0 && s.kp[p1]) v = cadd(v, B1[(size_t)r * KL + p1]);
                v = cscale(v, t);
            }
            X1[(size_t)r * KL + l] = v;
        }
    __syncthreads();
    // B' = (B1 W) Y into B1; (B1 W) G'_a2a2 into X2; A' = A1 + that (B1 W)^T
    dense_product<double, false, TCJ>(K1, Kb2, K2, X1, KL, X2, KL, B1, KL, s);
    dense_product<double, false, TCJ>(K1, K2, K2, X1, KL, B2, KL, X2, KL, s);
    acc_product<double, TCJ>(K1, K2, X2, X1, A1, KL, s);
    for (int e = threadIdx.x; e < Kb2 * Kb2; e += NT) {
        const int i = e / Kb2, l = e % Kb2;
        D1[(size_t)i * KL + l] = A2[(size_t)i * KL + l];
    }
    if constexpr (TCJ) {
        if (*(volatile int*)tst->ar.err()) flag |= 4;
    }
    __syncthreads();
    if (threadIdx.x == 0) *I1.flag = flag;
    __syncthreads();
}

// The interior domains joined, left to right, onto the left half in binary64.
// Joining domain d (columns ka .. kb, blocks A = G_aa, B = G_ab, D = g_b of the
// domain with its absorbing self-energy -i|t| at ka) to the system from the
// left lead up to column q = ka - 1 (E = its g at q, C = its corner block from
// the left lead's modes to q): the left part acts on column ka as W^T E W in
// place of the absorbing term, so with Sigma = W^T E W + i|t| (Dyson, Eq. 3)
//     G'_ab = (I - A Sigma)^-1 B = Y,     g'_b = D + B^T Sigma Y,
//     C'    = (C W) Y                     (G of the grown system from the lead
//                                          to kb; G_ba = B^T by symmetry).
// On return L.G = g'_b and L.P = C' of the last interior domain, in the working
// precision; L.X and the interior domains' buffers are scratch.  Returns the
// OR of the interior domains' flags and the joins' Gauss-Jordan flags.
template <class R, bool TCJ>
__device__ int join_interiors(const SweepArgs& a, const ChainDev& ch, const ChainCtx& c,
                              SweepSmem<double>& s, const Half<R>& L) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KL = c.KL;
    const double t = c.t, t2 = c.t2;
    zd* E = reinterpret_cast<zd*>(L.G);
    zd* C = reinterpret_cast<zd*>(L.P);
    zd* LX = reinterpret_cast<zd*>(L.X);
    int q = dom_bound(c.ncol, 1, a.ndom) - 1;
    int flag = 0;
    to_binary64<R>(L.G, col_size(c, q), col_size(c, q), KL);
    to_binary64<R>(L.P, KL, col_size(c, q), KL);
    // with more than one interior domain the tree of joins (tree_join_body)
    // has left all of them combined in domain 1's buffers, in binary64
    const bool tree = a.ndom > 3;
    const int dlast = tree ? 1 : a.ndom - 2;
    for (int d = 1; d <= dlast; ++d) {
        const Inner<R> I = inner_of<R>(a.ws, ch, d);
        const int ka = dom_bound(c.ncol, d, a.ndom);
        const int kb = dom_bound(c.ncol, tree ? a.ndom - 1 : d + 1, a.ndom) - 1;
        const int Ka = col_size(c, ka), Kb = col_size(c, kb), Kq = col_size(c, q), ct = ka & 3;
        flag |= *I.flag;
        if (!tree) {
            to_binary64<R>(I.A, Ka, Ka, KL);
            to_binary64<R>(I.P, Ka, Kb, KL);
            to_binary64<R>(I.G, Kb, Kb, KL);
        }
        zd* A = reinterpret_cast<zd*>(I.A);
        zd* B = reinterpret_cast<zd*>(I.P);
        zd* D = reinterpret_cast<zd*>(I.G);
        zd* IX = reinterpret_cast<zd*>(I.X);
        load_col(c, ka, s.kc, nullptr);
        load_col(c, q, s.kp, nullptr);
        __syncthreads();
        // Sigma = t^2 S^T E S on column ka (kept atoms only) into LX
        for (int i = warp; i < Ka; i += NWARP) {
            int a0, a1;
            col_src(ct, i, Kq, a0, a1);
            const bool ki = s.kc[i];
            const bool ka0 = a0 >= 0 && s.kp[a0], ka1 = a1 >= 0 && s.kp[a1];
            for (int l = lane; l < Ka; l += 32) {
                zd v = {0.0, 0.0};
                if (ki && s.kc[l]) {
                    int b0, b1;
                    col_src(ct, l, Kq, b0, b1);
                    const bool kb0 = b0 >= 0 && s.kp[b0], kb1 = b1 >= 0 && s.kp[b1];
                    if (ka0 && kb0) v = cadd(v, E[(size_t)a0 * KL + b0]);
                    if (ka0 && kb1) v = cadd(v, E[(size_t)a0 * KL + b1]);
                    if (ka1 && kb0) v = cadd(v, E[(size_t)a1 * KL + b0]);
                    if (ka1 && kb1) v = cadd(v, E[(size_t)a1 * KL + b1]);
                    v = cscale(v, t2);
                }
                if (i == l && ki) v.im += fabs(t);      // the absorbing term taken out
                LX[(size_t)i * KL + l] = v;
            }
        }
        __syncthreads();
        // X = I - A Sigma into IX; B^T Sigma into A (A read for the last time)
        dense_product<double, false, TCJ>(Ka, Ka, Ka, A, KL, LX, KL, IX, KL, s);
        for (int e = threadIdx.x; e < Ka * Ka; e += NT) {
            const int i = e / Ka, l = e % Ka;
            zd& x = IX[(size_t)i * KL + l];
            x = {((i == l) ? 1.0 : 0.0) - x.re, -x.im};
        }
        __syncthreads();
        dense_product<double, true, TCJ>(Kb, Ka, Ka, B, KL, LX, KL, A, KL, s);
        // X^-1 into LX, Y = X^-1 B into IX
        const double amax2 = max_abs2(IX, Ka, KL, s.red);
        flag |= cta_gj_invert<double, TCJ>(IX, Ka, KL, LX, KL, s.gj, amax2);
        dense_product<double, false, TCJ>(Ka, Kb, Ka, LX, KL, B, KL, IX, KL, s);
        // g'_b = D + (B^T Sigma) Y into E
        dense_product<double, false, TCJ>(Kb, Kb, Ka, A, KL, IX, KL, E, KL, s);
        for (int e = threadIdx.x; e < Kb * Kb; e += NT) {
            const int i = e / Kb, l = e % Kb;
            E[(size_t)i * KL + l] = cadd(E[(size_t)i * KL + l], D[(size_t)i * KL + l]);
        }
        // C W (KL x Ka) into LX, then C' = (C W) Y into C
        for (int r = warp; r < KL; r += NWARP)
            for (int l = lane; l < Ka; l += 32) {
                zd v = {0.0, 0.0};
                if (s.kc[l]) {
                    int a0, a1;
                    col_src(ct, l, Kq, a0, a1);
                    if (a0 >= 0 && s.kp[a0]) v = cadd(v, C[(size_t)r * KL + a0]);
                    if (a1 >= 0 && s.kp[a1]) v = cadd(v, C[(size_t)r * KL + a1]);
                    v = cscale(v, t);
                }
                LX[(size_t)r * KL + l] = v;
            }
        __syncthreads();
        dense_product<double, false, TCJ>(KL, Kb, Ka, LX, KL, IX, KL, C, KL, s);
        q = kb;
    }
    to_working<R>(L.G, col_size(c, q), col_size(c, q), KL);
    to_working<R>(L.P, KL, col_size(c, q), KL);
    return flag;
}

// The Dyson step across the bond between columns m-1 and m of chain ci, in
// binary64, and the trace; writes T and the status word.  Scratch: the two
// halves' X and, once read, their G and P.  bm: the launch's panel width.
// TCJ (chains of more than two domains in a tensor-core precision): the
// joins' products and inverses' rank-b updates on the tensor cores, sliced
// from binary64 and summed in binary64 (the block holds TMEM, tst).
// Every thread; ends with a barrier.
template <class R, bool TCJ = false>
__device__ __noinline__ void merge_body(const SweepArgs a, int ci, int bm, tc::State* tst = nullptr) {
    SweepSmem<double> s = carve<double>(rgf_dyn_smem, a.Kmax, TCJ, bm);
    if constexpr (TCJ) {
        s.gj.tcs = tst;
        s.tcs = tst;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const ChainDev& ch = a.chains[ci];
    const int lst = lead_state(a.lead_status, ch.lead);
    if (lst != ST_OK) {
        if (threadIdx.x == 0) {
            a.T[ci] = NAN;
            if (a.status) a.status[ci] = lst;
        }
        __syncthreads();
        return;
    }
    const ChainCtx c = make_ctx(ch, a.leads[ch.lead], a.leadout, a.eta_d, 0);
    const Half<R> L = half_of<R>(a.ws, ch, 0), Rt = half_of<R>(a.ws, ch, 1);
    int flag = *L.flag | *Rt.flag;
    int m = left_cols(c.ncol);
    if (a.ndom > 2) {
        flag |= join_interiors<R, TCJ>(a, ch, c, s, L);
        m = dom_bound(c.ncol, a.ndom - 1, a.ndom);
    }
    const int KL = c.KL, KR = c.KR;
    const int K = col_size(c, m), Kp = col_size(c, m - 1), ct = m & 3;
    load_col(c, m, s.kc, nullptr);
    load_col(c, m - 1, s.kp, nullptr);
    __syncthreads();
    zd* XL = reinterpret_cast<zd*>(L.X);
    zd* XR = reinterpret_cast<zd*>(Rt.X);
    zd* GLd = reinterpret_cast<zd*>(L.G);
    zd* GRd = reinterpret_cast<zd*>(Rt.G);
    zd* PRd = reinterpret_cast<zd*>(Rt.P);
    const double t = c.t, t2 = c.t2;
    // SigmaL_m = t^2 S^T gl_{m-1} S (kept atoms only) into XL
    for (int i = warp; i < K; i += NWARP) {
        int a0, a1;
        col_src(ct, i, Kp, a0, a1);
        const bool ki = s.kc[i];
        const bool ka0 = a0 >= 0 && s.kp[a0], ka1 = a1 >= 0 && s.kp[a1];
        for (int l = lane; l < K; l += 32) {
            zd v = {0.0, 0.0};
            if (ki && s.kc[l]) {
                int b0, b1;
                col_src(ct, l, Kp, b0, b1);
                const bool kb0 = b0 >= 0 && s.kp[b0], kb1 = b1 >= 0 && s.kp[b1];
                if (ka0 && kb0) v = cadd(v, to_z(L.G[(size_t)a0 * KL + b0]));
                if (ka0 && kb1) v = cadd(v, to_z(L.G[(size_t)a0 * KL + b1]));
                if (ka1 && kb0) v = cadd(v, to_z(L.G[(size_t)a1 * KL + b0]));
                if (ka1 && kb1) v = cadd(v, to_z(L.G[(size_t)a1 * KL + b1]));
                v = cscale(v, t2);
            }
            XL[(size_t)i * KL + l] = v;
        }
    }
    __syncthreads();
    // X = I - gr_m SigmaL_m into XR, its inverse into XL
    to_binary64<R>(Rt.G, K, K, KL);
    dense_product<double, false, TCJ>(K, K, K, GRd, KL, XL, KL, XR, KL, s);
    for (int e = threadIdx.x; e < K * K; e += NT) {
        const int i = e / K, l = e % K;
        zd& x = XR[(size_t)i * KL + l];
        x = {((i == l) ? 1.0 : 0.0) - x.re, -x.im};
    }
    __syncthreads();
    const double amax2 = max_abs2(XR, K, KL, s.red);
    flag |= cta_gj_invert<double, TCJ>(XR, K, KL, XL, KL, s.gj, amax2);
    // Y = Pl_{m-1} W_m (KL x K) into GL (gl no longer needed), then
    // Y (I - gr SigmaL)^-1 into XR and its product with Pr_m^T into GL
    for (int r = warp; r < KL; r += NWARP)
        for (int l = lane; l < K; l += 32) {
            zd v = {0.0, 0.0};
            if (s.kc[l]) {
                int a0, a1;
                col_src(ct, l, Kp, a0, a1);
                if (a0 >= 0 && s.kp[a0]) v = cadd(v, to_z(L.P[(size_t)r * KL + a0]));
                if (a1 >= 0 && s.kp[a1]) v = cadd(v, to_z(L.P[(size_t)r * KL + a1]));
                v = cscale(v, t);
            }
            GLd[(size_t)r * KL + l] = v;
        }
    __syncthreads();
    dense_product<double, false, TCJ>(KL, K, K, GLd, KL, XL, KL, XR, KL, s);
    to_binary64<R>(Rt.P, KR, K, KL);
    cta_gemm<double, false, true>(KL, KR, K, XR, KL, PRd, KL, GLd, KL, GEMM_SET, s.gemm);
    // T = sum_pq gamma_p gamma'_q |P_pq|^2
    double acc = 0.0;
    const zd* w = c.w();
    for (int e = threadIdx.x; e < KL * KR; e += NT) {
        const int p = e / KR, q = e % KR;
        const zd v = GLd[(size_t)p * KL + q];
        acc += (-2.0 * w[p].im) * (-2.0 * w[q].im) * (v.re * v.re + v.im * v.im);
    }
    if constexpr (TCJ) {
        if (*(volatile int*)tst->ar.err()) flag |= 4;
    }
    const double T = block_sum(acc, s.red);
    if (threadIdx.x == 0) {
        const int st = chain_status(c, flag, T);
        a.T[ci] = (st == ST_OK) ? T : NAN;
        if (a.status) a.status[ci] = st;
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Launch helpers
// ---------------------------------------------------------------------------
template <class K>
cudaError_t set_smem(K kern, size_t smem) {
    return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Precisions: 0 RGF_FP64, 1 RGF_MIXED, 2 RGF_MIXED_TC, 3 RGF_FP64_TC.
bool uses_tc(int precision) { return precision == 2 || precision == 3; }
bool binary64(int precision) { return precision == 0 || precision == 3; }

// Panel width of a launch of `precision` and the shared memory of its
// binary64 steps and of its recursion.
int launch_panel(int precision, int Kmax) { return gj_panel_width(Kmax, uses_tc(precision)); }
size_t f64_smem(int precision, int Kmax) {
    return sweep_total_bytes(Kmax, launch_panel(precision, Kmax), false);
}
size_t rec_smem(int precision, int Kmax) {
    const size_t b = sweep_total_bytes(Kmax, launch_panel(precision, Kmax), uses_tc(precision));
    // a tensor-core block holds all 512 TMEM columns: ask for more than half
    // of an SM's shared memory so that no second block shares its SM (the
    // register file already allows only one)
    return uses_tc(precision) && b < 120 * 1024 ? 120 * 1024 : b;
}

SweepArgs make_args(const ChainDev* chains, const int* order, int nchains, int Kmax,
                    double eta_device, const void* leadout, const int* lead_status,
                    const LeadDev* leads, void* ws, double* T, int32_t* status, int ndom = 2) {
    return SweepArgs{chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status,
                     leads, ws, T, status, ndom};
}

}  // namespace
}  // namespace rgf
