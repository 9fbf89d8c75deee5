// rgf_grad.cu -- dT/d eps for every on-site energy, one thread block per
// chain, over the column slices of rgf_half.cuh.
//
// The paper does not differentiate; the derivative follows from Eq. 1 and
// Eq. 2.  With A = z - H - Sigma and dA/d eps_i = -e_i e_i^T, dG = G e_i e_i^T G,
// so for T = Tr[Gamma_L G_1L Gamma_R G_1L^dagger]:
//
//   dT/d eps_i = 2 Re (G_kL M G_1k)_ii,   M = Gamma_R G_1L^dagger Gamma_L,
//
// for site i of column k.  The blocks of the whole system's G come from the
// Dyson equation (Eq. 3) with the bond on either side of column k cut:
//
//   G_kk = (A_k - W_k^T gl_{k-1} W_k - W_{k+1} gr_{k+1} W_{k+1}^T)^-1
//   G_1k = Pl_{k-1} W_k G_kk,          G_kL = G_kk W_{k+1} Qr_{k+1}
//
// gl_k, Pl_k = G_1k of the columns left of the cut (the recursion of Eqs. 4-5,
// as in the forward sweep) and gr_k, Qr_k = G_kL of the columns right of it
// (the same recursion from the right lead).  This two-sided form keeps its
// accuracy next to the poles of the half systems (E near 0), where a reverse
// sweep through the gl_k amplifies rounding at isolated sites.
//
// Passes: the right-to-left recursion stores (gr, Qr) at the end of every
// segment of seg_cols columns and yields G_1L = Qr_0, T and M; the
// left-to-right pass recomputes each segment's (gr, Qr) from its checkpoint,
// then walks it forwards carrying gl, Pl and forming G_kk, G_1k, G_kL and the
// gradient of each column; T comes from the left recursion, as in the
// forward sweep.  With TC (precision RGF_MIXED_TC) the dense
// products run on the tcgen05 tensor cores (rgf_tc.cuh); the block holds the
// SM's TMEM for the whole launch.
//
// The same pass yields the local density of states rho_i(E) = -Im (G_kk)_ii / pi
// (the paper notes that the Green's function of Eq. 1 gives the charge density;
// rho is its integrand over energy): `out_mode` selects the gradient
// (OUT_GRAD), rho (OUT_LDOS), or both into two arrays; with rho alone the
// products that only the gradient needs (G_1k, G_kL and the trace with M) are
// skipped.
#include "rgf_steps.cuh"

namespace rgf {

namespace {

constexpr double kInvPi = 0.318309886183790671537767526745;   // 1 / pi

template <class R>
__device__ void copy_blk(cx<R>* D, const cx<R>* S, size_t n) {
    for (size_t e = threadIdx.x; e < n; e += NT) D[e] = S[e];
    __syncthreads();
}

// X = (z - eps_k) I - [left] SigmaL_k - [right] SigmaR_k for column k, identity
// rows and columns at removed atoms.  SigmaL_k: Sigma_L at k = 0, else
// W_k^T glp W_k; SigmaR_k: Sigma_R at the last column, else
// W_{k+1} grn W_{k+1}^T (W = t times the bond pattern between two columns,
// applied as a stencil).  Needs s.kc, s.eps of column k, s.kp of k-1 and s.kn
// of k+1.  Returns max |X_il|^2 over the block (ends with a barrier).
template <class R>
__device__ double build_A(const ChainCtx& c, int k, bool left, const cx<R>* glp, bool right,
                          const cx<R>* grn, cx<R>* X, SweepSmem<R>& s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KL = c.KL, ct = k & 3, K = col_size(c, k);
    const bool first = k == 0, last = k == c.ncol - 1;
    const int Kp = first ? 0 : col_size(c, k - 1), Kn = last ? 0 : col_size(c, k + 1);
    const int ctn = (k + 1) & 3;
    const auto t2 = Hop<R>::t2(c);
    double amax2 = 0.0;
    for (int i = warp; i < K; i += NWARP) {
        int a0 = -1, a1 = -1, n0 = -1, n1 = -1;
        if (left && !first) col_src(ct, i, Kp, a0, a1);
        if (right && !last) col_src_T(ctn, i, Kn, n0, n1);
        const bool ki = s.kc[i];
        const bool ka0 = a0 >= 0 && s.kp[a0], ka1 = a1 >= 0 && s.kp[a1];
        const bool kn0 = n0 >= 0 && s.kn[n0], kn1 = n1 >= 0 && s.kn[n1];
        for (int l = lane; l < K; l += 32) {
            cx<R> v;
            if (!ki || !s.kc[l]) {
                v = (i == l) ? from_z<R>(1.0, 0.0) : czero<R>();
            } else {
                // the left term as the forward sweep forms it (inv_column), so
                // that the left recursion reproduces the forward sweep bit for bit
                cx<R> sig = czero<R>();
                if (left && first) sig = ld_z<R>(c.SigL() + (size_t)i * KL + l);
                if (left && !first) {
                    int b0, b1;
                    col_src(ct, l, Kp, b0, b1);
                    const bool kb0 = b0 >= 0 && s.kp[b0], kb1 = b1 >= 0 && s.kp[b1];
                    if (ka0 && kb0) sig = cadd(sig, glp[(size_t)a0 * KL + b0]);
                    if (ka0 && kb1) sig = cadd(sig, glp[(size_t)a0 * KL + b1]);
                    if (ka1 && kb0) sig = cadd(sig, glp[(size_t)a1 * KL + b0]);
                    if (ka1 && kb1) sig = cadd(sig, glp[(size_t)a1 * KL + b1]);
                    sig = cscale(sig, t2);
                }
                if (right && last) sig = cadd(sig, ld_z<R>(c.SigR() + (size_t)i * c.KR + l));
                if (right && !last) {
                    int m0, m1;
                    col_src_T(ctn, l, Kn, m0, m1);
                    const bool km0 = m0 >= 0 && s.kn[m0], km1 = m1 >= 0 && s.kn[m1];
                    cx<R> w = czero<R>();
                    if (kn0 && km0) w = cadd(w, grn[(size_t)n0 * KL + m0]);
                    if (kn0 && km1) w = cadd(w, grn[(size_t)n0 * KL + m1]);
                    if (kn1 && km0) w = cadd(w, grn[(size_t)n1 * KL + m0]);
                    if (kn1 && km1) w = cadd(w, grn[(size_t)n1 * KL + m1]);
                    sig = cadd(sig, cscale(w, t2));
                }
                v = (i == l) ? from_z<R>(c.z.re - s.eps[i], c.z.im) : czero<R>();
                v = csub(v, sig);
            }
            X[(size_t)i * KL + l] = v;
            const double a2 = (double)cabs2f(v);
            amax2 = (a2 > amax2 || isnan(a2)) ? a2 : amax2;
        }
    }
    return block_max(amax2, s.red);
}

// Column k's matrix (build_A) inverted into Gout; one out-of-line copy for
// the four call sites.  Returns the Gauss-Jordan flags.
template <class R, bool TC64>
static __device__ __noinline__ int build_invert(const ChainCtx& c, int k, bool left, const cx<R>* glp,
                                                bool right, const cx<R>* grn, cx<R>* X, cx<R>* Gout,
                                                SweepSmem<R>& s) {
    const double amax2 = build_A<R>(c, k, left, glp, right, grn, X, s);
    return cta_gj_invert<R, TC64>(X, col_size(c, k), c.KL, Gout, c.KL, s.gj, amax2);
}

// Y = Pl W_k (KL x K): Y[r][l] = t sum over the kept sources a of l in column
// k-1 of Pl[r][a]; zero for a removed l.  Ends with a barrier.
template <class R>
__device__ void stencil_left(const ChainCtx& c, int k, const cx<R>* Pl, cx<R>* Y, SweepSmem<R>& s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KL = c.KL, ct = k & 3, K = col_size(c, k), Kp = col_size(c, k - 1);
    const auto t = Hop<R>::t(c);
    for (int r = warp; r < KL; r += NWARP)
        for (int l = lane; l < K; l += 32) {
            cx<R> v = czero<R>();
            if (s.kc[l]) {
                int a0, a1;
                col_src(ct, l, Kp, a0, a1);
                if (a0 >= 0 && s.kp[a0]) v = cadd(v, Pl[(size_t)r * KL + a0]);
                if (a1 >= 0 && s.kp[a1]) v = cadd(v, Pl[(size_t)r * KL + a1]);
                v = cscale(v, t);
            }
            Y[(size_t)r * KL + l] = v;
        }
    __syncthreads();
}

// Z = W_{k+1} Qr (K x KR): Z[a][q] = t sum over the kept partners i of a in
// column k+1 of Qr[i][q]; zero for a removed a.  Ends with a barrier.
template <class R>
__device__ void stencil_right(const ChainCtx& c, int k, const cx<R>* Qr, cx<R>* Z, SweepSmem<R>& s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int KL = c.KL, KR = c.KR, K = col_size(c, k), Kn = col_size(c, k + 1);
    const int ctn = (k + 1) & 3;
    const auto t = Hop<R>::t(c);
    for (int a = warp; a < K; a += NWARP) {
        int n0 = -1, n1 = -1;
        if (s.kc[a]) col_src_T(ctn, a, Kn, n0, n1);
        const bool k0 = n0 >= 0 && s.kn[n0], k1 = n1 >= 0 && s.kn[n1];
        for (int q = lane; q < KR; q += 32) {
            cx<R> v = czero<R>();
            if (k0) v = cadd(v, Qr[(size_t)n0 * KL + q]);
            if (k1) v = cadd(v, Qr[(size_t)n1 * KL + q]);
            Z[(size_t)a * KL + q] = cscale(v, t);
        }
    }
    __syncthreads();
}

// Masks and on-site energies of column k and its neighbours into shared memory.
template <class R>
__device__ void load_cols(const ChainCtx& c, int k, SweepSmem<R>& s) {
    load_col(c, k, s.kc, s.eps);
    load_col(c, k - 1, s.kp, nullptr);
    load_col(c, k + 1, s.kn, nullptr);
    __syncthreads();
}

}  // namespace

template <class R, bool TC>
__global__ void __launch_bounds__(NT, 1)
grad_kernel(const ChainDev* __restrict__ chains, const int* __restrict__ order, int nchains,
            int Kmax, double eta_d, const zd* __restrict__ leadout,
            const int* __restrict__ lead_status, const LeadDev* __restrict__ leads,
            cx<R>* __restrict__ ws, const int* __restrict__ seg_cols, double* __restrict__ Tout,
            double* __restrict__ dT, double* __restrict__ rho, int out_mode,
            int32_t* __restrict__ status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SweepSmem<R> s = carve<R>(smem_raw, Kmax, TC);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int ci = order[blockIdx.x];
    const ChainDev ch = chains[ci];
    const int lst = lead_state(lead_status, ch.lead);
    if (lst != ST_OK) {
        if (threadIdx.x == 0) { Tout[ci] = NAN; if (status) status[ci] = lst; }
        return;
    }
    const ChainCtx c = make_ctx(ch, leads[ch.lead], leadout, eta_d);
    const int KL = c.KL, KR = c.KR, ncol = c.ncol;
    const int Sc = seg_cols[ci];
    const int nseg = (ncol + Sc - 1) / Sc;
    const size_t B = (size_t)KL * KL;
    cx<R>* base = ws + ch.ws_off;
    cx<R> *X = base, *Y = base + B, *Z = base + 2 * B, *U = base + 3 * B;
    cx<R> *Gkk = base + 4 * B, *G1k = base + 5 * B, *GkL = base + 6 * B;
    cx<R> *gl = base + 7 * B, *Pl = base + 8 * B, *Mb = base + 9 * B;
    cx<R> *GL = base + 10 * B, *GR = base + 11 * B, *gr = base + 12 * B, *Qr = base + 13 * B;
    cx<R>* ckpt = base + 14 * B;                       // (gr, Qr) at column (j + 1) Sc
    cx<R>* seg = ckpt + (size_t)nseg * 2 * B;          // (Sc + 1) x (gr, Qr)
    const bool want_grad = (out_mode & OUT_GRAD) != 0, want_ldos = (out_mode & OUT_LDOS) != 0;
    double* grad = want_grad ? dT + ch.grad_off : nullptr;
    double* ldos = want_ldos ? rho + ch.grad_off : nullptr;
    tc::State tst;
    if constexpr (TC) tc_attach<R>(Kmax, s, tst);

    // Right-to-left recursion: gr_k = (A_k - W_{k+1} gr_{k+1} W_{k+1}^T)^-1
    // (Sigma_R at the last column, Sigma_L at column 0), Qr_k = gr_k W_{k+1} Qr_{k+1}.
    int flag = 0;
    for (int k = ncol - 1; k >= 0; --k) {
        load_cols(c, k, s);
        const int K = col_size(c, k);
        flag |= build_invert<R, TC>(c, k, k == 0, nullptr, true, gr, X, gr, s);
        if (k == ncol - 1) {
            copy_blk(Qr, gr, B);
        } else {
            stencil_right<R>(c, k, Qr, Z, s);
            dense_product<R, false, TC>(K, KR, K, gr, KL, Z, KL, Qr, KL, s);
        }
        if (k > 0 && k % Sc == 0) {
            cx<R>* cp = ckpt + (size_t)(k / Sc - 1) * 2 * B;
            copy_blk(cp, gr, B);
            copy_blk(cp + B, Qr, B);
        }
    }
    if constexpr (TC) {
        if (*(volatile int*)tst.ar.err()) flag |= 4;
    }
    // G_1L = Qr_0 (KL x KR).  A chain that fails here stops; the T reported
    // for the others comes from the left recursion below (the forward
    // sweep's arithmetic).
    {
        const double Tr = trace_T<R>(c, Qr, X, Z, U, s);
        const int st = chain_status(c, flag, Tr);
        if (st != ST_OK) {
            if (threadIdx.x == 0) {
                Tout[ci] = NAN;
                if (status) status[ci] = st;
            }
            if constexpr (TC) tc::teardown(tst.ar);
            return;
        }
    }

    // M = Gamma_R G_1L^dagger Gamma_L  (KR x KL)
    for (size_t e = threadIdx.x; e < B && want_grad; e += NT) {
        GL[e] = ld_z<R>(c.GamL() + e);                              // KL x KL, ld KL
        if (e < (size_t)KR * KR) GR[e] = ld_z<R>(c.GamR() + e);     // KR x KR, ld KR
        const int b = (int)(e / KL), a = (int)(e % KL);
        if (b < KR) Y[e] = cconj(Qr[(size_t)a * KL + b]);         // Y[b][a] = conj(G_1L[a][b])
    }
    __syncthreads();
    if (want_grad) {
        dense_product<R, false, TC>(KR, KL, KR, GR, KR, Y, KL, U, KL, s);
        dense_product<R, false, TC>(KR, KL, KL, U, KL, GL, KL, Mb, KL, s);
    }

    // Left-to-right pass, segment by segment.
    for (int j = 0; j < nseg; ++j) {
        const int k0 = j * Sc, k1 = min(ncol, k0 + Sc);
        // (gr, Qr) of columns k0 .. k1 - 1 from the checkpoint at k1
        if (k1 < ncol) {
            cx<R>* cp = ckpt + (size_t)j * 2 * B;
            cx<R>* sl = seg + (size_t)(k1 - k0) * 2 * B;
            copy_blk(sl, cp, B);
            copy_blk(sl + B, cp + B, B);
        }
        for (int k = k1 - 1; k >= k0; --k) {
            cx<R>* sk = seg + (size_t)(k - k0) * 2 * B;
            const cx<R>* sn = sk + 2 * B;
            load_cols(c, k, s);
            const int K = col_size(c, k);
            flag |= build_invert<R, TC>(c, k, k == 0, nullptr, true, sn, X, sk, s);
            if (k == ncol - 1) {
                copy_blk(sk + B, sk, B);
            } else {
                stencil_right<R>(c, k, sn + B, Z, s);
                dense_product<R, false, TC>(K, KR, K, sk, KL, Z, KL, sk + B, KL, s);
            }
        }
        for (int k = k0; k < k1; ++k) {
            const cx<R>* sn = seg + (size_t)(k - k0 + 1) * 2 * B;   // (gr, Qr)_{k+1}
            const int ct = k & 3, K = col_size(c, k);
            (void)ct;
            const bool last = k == ncol - 1;
            load_cols(c, k, s);
            // G_kk
            flag |= build_invert<R, TC>(c, k, true, gl, true, sn, X, Gkk, s);
            const int n = k >> 2;
            if (want_ldos) {
                // rho_i = -Im (G_kk)_ii / pi; 0 on removed atoms
                for (int i = threadIdx.x; i < K; i += NT)
                    ldos[(size_t)n * c.M + 4 * i + ct] =
                        s.kc[i] ? -to_z(Gkk[(size_t)i * KL + i]).im * kInvPi : 0.0;
            }
            if (k > 0) stencil_left<R>(c, k, Pl, Y, s);     // Y = Pl_{k-1} W_k
            if (want_grad) {
                // G_1k = Pl_{k-1} W_k G_kk  (KL x K)
                const cx<R>* g1 = Gkk;
                if (k > 0) {
                    dense_product<R, false, TC>(KL, K, K, Y, KL, Gkk, KL, G1k, KL, s);
                    g1 = G1k;
                }
                // G_kL = G_kk W_{k+1} Qr_{k+1}  (K x KR)
                const cx<R>* gL = Gkk;
                if (!last) {
                    stencil_right<R>(c, k, sn + B, Z, s);
                    dense_product<R, false, TC>(K, KR, K, Gkk, KL, Z, KL, GkL, KL, s);
                    gL = GkL;
                }
                // dT/d eps_i = 2 Re sum_b (G_kL M)[i][b] G_1k[b][i]
                dense_product<R, false, TC>(K, KL, KR, gL, KL, Mb, KL, U, KL, s);
                for (int i = warp; i < K; i += NWARP) {
                    double acc = 0.0;
                    for (int b = lane; b < KL; b += 32) {
                        const zd u = to_z(U[(size_t)i * KL + b]), g = to_z(g1[(size_t)b * KL + i]);
                        acc += u.re * g.re - u.im * g.im;
                    }
                    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
                    if (lane == 0 && s.kc[i]) grad[(size_t)n * c.M + 4 * i + ct] = 2.0 * acc;
                }
            }
            // gl_k and Pl_k (the forward recursion)
            flag |= build_invert<R, TC>(c, k, true, gl, last, nullptr, X, gl, s);
            if (k == 0) copy_blk(Pl, gl, B);
            else dense_product<R, false, TC>(KL, K, K, Y, KL, gl, KL, Pl, KL, s);
        }
    }
    if constexpr (TC) {
        if (*(volatile int*)tst.ar.err()) flag |= 4;
    }
    // T from Pl = G_1L of the left recursion
    const double T = trace_T<R>(c, Pl, X, Z, U, s);
    const int st = chain_status(c, flag, T);
    if (threadIdx.x == 0) {
        Tout[ci] = (st == ST_OK) ? T : NAN;
        if (status) status[ci] = st;
    }
    if constexpr (TC) tc::teardown(tst.ar);
}

size_t grad_ws_elems(int N, int L, int seg_cols) {
    size_t KL = (size_t)col_KL(N);
    size_t ncol = 4 * (size_t)L;
    size_t nseg = (ncol + seg_cols - 1) / seg_cols;
    return (14 + 2 * nseg + 2 * ((size_t)seg_cols + 1)) * KL * KL;
}

cudaError_t launch_grad(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, const int* seg_cols, double* T, double* dT,
                        double* rho, int out_mode, int32_t* status, cudaStream_t st) {
    if (nchains <= 0) return cudaSuccess;
    // the _TC precisions on the pipes where the tensor-core layout does not fit
    if ((precision == 2 || precision == 3) && !tc_layout_fits(Kmax)) precision = precision == 2 ? 1 : 0;
    const bool tc = precision == 2 || precision == 3;
    const size_t smem = sweep_smem_bytes(Kmax, tc);
    cudaError_t e;
    if (precision == 3) {
        e = cudaFuncSetAttribute(grad_kernel<double, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        grad_kernel<double, true><<<nchains, NT, smem, st>>>(
            chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status, leads,
            (zd*)ws, seg_cols, T, dT, rho, out_mode, status);
    } else if (precision == 0) {
        e = cudaFuncSetAttribute(grad_kernel<double, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        grad_kernel<double, false><<<nchains, NT, smem, st>>>(
            chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status, leads,
            (zd*)ws, seg_cols, T, dT, rho, out_mode, status);
    } else if (tc) {
        e = cudaFuncSetAttribute(grad_kernel<df32, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        grad_kernel<df32, true><<<nchains, NT, smem, st>>>(
            chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status, leads,
            (zf*)ws, seg_cols, T, dT, rho, out_mode, status);
    } else {
        e = cudaFuncSetAttribute(grad_kernel<df32, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        grad_kernel<df32, false><<<nchains, NT, smem, st>>>(
            chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status, leads,
            (zf*)ws, seg_cols, T, dT, rho, out_mode, status);
    }
    return cudaGetLastError();
}

}  // namespace rgf
