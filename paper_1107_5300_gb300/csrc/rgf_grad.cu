// rgf_grad.cu -- dT/d eps for every on-site energy: the adjoint (reverse-mode)
// sweep of the column recursion in rgf_sweep.cu, one thread block per chain.
//
// The paper does not differentiate; the derivative follows from Eq. 1 and
// Eq. 2.  With X_bar = dT/dX (holomorphic part, dT = 2 Re Tr[X_bar^T dX]) and
// the slice Green's functions g_k complex symmetric (H real symmetric):
//
//   P_bar_last = Gamma_L conj(P_last) Gamma_R
//   for k = last .. 0:
//     g_bar_k  = [k > 0]  W_k^T P_{k-1}^T P_bar_k      (strip P_k = P_{k-1} W_k g_k)
//              + [k = 0]  P_bar_0                      (P_0 = g_0)
//              - [k < last] W_{k+1} A_bar_{k+1} W_{k+1}^T   (A_{k+1} = ... - W^T g_k W)
//     A_bar_k  = -g_k g_bar_k g_k                      (g_k = A_k^-1)
//     dT/d eps_{k,i} = -2 Re (A_bar_k)_ii             (A_k = z - eps_k - ...)
//     P_bar_{k-1} = P_bar_k g_k W_k^T
//
// Memory: the forward pass stores (g, P) at the start of every segment of
// 4 * stride columns (stride in unit cells, ~sqrt(L) by default); the reverse
// pass recomputes each segment's g_k, P_k from its checkpoint, then walks it
// backwards.  The workspace holds Q = -A_bar (so dT/d eps_i = 2 Re Q_ii).
// With TC (precision RGF_MIXED_TC) the forward and recomputed column steps
// and the dense products of the reverse pass run on the tcgen05 tensor cores
// (rgf_tc.cuh); the block holds the SM's TMEM for the whole launch.
#include "rgf_steps.cuh"

namespace rgf {

namespace {

template <class R>
__device__ void copy_blk(cx<R>* D, const cx<R>* S, size_t n) {
    for (size_t e = threadIdx.x; e < n; e += NT) D[e] = S[e];
    __syncthreads();
}

}  // namespace

template <class R, bool TC>
__global__ void __launch_bounds__(NT, 1)
grad_kernel(const ChainDev* __restrict__ chains, const int* __restrict__ order, int nchains,
            int Kmax, double eta_d, const zd* __restrict__ leadout,
            const int* __restrict__ lead_status, const LeadDev* __restrict__ leads,
            cx<R>* __restrict__ ws, const int* __restrict__ seg_cols, double* __restrict__ Tout,
            double* __restrict__ dT, int32_t* __restrict__ status) {
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
    cx<R> *X = base, *Y = base + B, *G = base + 2 * B, *P = base + 3 * B;
    cx<R>* Pb[2] = {base + 4 * B, base + 5 * B};
    cx<R>* Qb[2] = {base + 6 * B, base + 7 * B};
    cx<R> *gbar = base + 8 * B, *T1 = base + 9 * B, *GL = base + 10 * B, *GR = base + 11 * B;
    cx<R>* ckpt = base + 12 * B;                       // nseg x (g, P)
    cx<R>* seg = ckpt + (size_t)nseg * 2 * B;          // (Sc + 1) x (g, P)
    double* grad = dT + ch.grad_off;
    const auto t = Hop<R>::t(c);
    const auto t2 = Hop<R>::t2(c);
    tc::State tst;
    if constexpr (TC) tc_attach<R>(Kmax, s, tst);

    // Forward pass with checkpoints.
    int flag = 0;
    for (int k = 0; k < ncol; ++k) {
        if (k > 0 && k % Sc == 0) {
            const int j = k / Sc;
            copy_blk(ckpt + (size_t)j * 2 * B, G, B);
            copy_blk(ckpt + (size_t)j * 2 * B + B, P, B);
        }
        load_col(c, k, s.kc, s.eps);
        load_col(c, k - 1, s.kp, nullptr);
        __syncthreads();
        flag |= fwd_column<R>(c, k, G, G, P, P, X, Y, s);
    }
    if constexpr (TC) {
        if (*(volatile int*)tst.ar.err()) flag |= 4;
    }
    const double T = trace_T<R>(c, P, X, T1, gbar, s);
    const int st = chain_status(c, flag, T);
    if (threadIdx.x == 0) {
        Tout[ci] = (st == ST_OK) ? T : NAN;
        if (status) status[ci] = st;
    }
    if (st != ST_OK) {
        if constexpr (TC) tc::teardown(tst.ar);
        return;
    }

    // P_bar = Gamma_L conj(P) Gamma_R  (KL x KR)
    for (size_t e = threadIdx.x; e < B; e += NT) {
        GL[e] = ld_z<R>(c.GamL + e);                      // KL x KL, ld KL
        if (e < (size_t)KR * KR) GR[e] = ld_z<R>(c.GamR + e);   // KR x KR, ld KR
        if ((int)(e % KL) < KR) Y[e] = cconj(P[e]);
    }
    __syncthreads();
    dense_product<R, false>(KL, KR, KL, GL, KL, Y, KL, T1, KL, s);
    dense_product<R, false>(KL, KR, KR, T1, KL, GR, KR, Pb[0], KL, s);
    int pb = 0, qb = 0;

    for (int j = nseg - 1; j >= 0; --j) {
        const int k0 = j * Sc, k1 = min(ncol, k0 + Sc);
        if (j > 0) {
            copy_blk(seg, ckpt + (size_t)j * 2 * B, B);
            copy_blk(seg + B, ckpt + (size_t)j * 2 * B + B, B);
        }
        for (int k = k0; k < k1; ++k) {
            cx<R>* sp = seg + (size_t)(k - k0) * 2 * B;
            cx<R>* sn = sp + 2 * B;
            load_col(c, k, s.kc, s.eps);
            load_col(c, k - 1, s.kp, nullptr);
            __syncthreads();
            fwd_column<R>(c, k, sp, sn, sp + B, sn + B, X, Y, s);
        }
        for (int k = k1 - 1; k >= k0; --k) {
            const cx<R>* gk = seg + (size_t)(k - k0 + 1) * 2 * B;
            const cx<R>* Pm = seg + (size_t)(k - k0) * 2 * B + B;   // P_{k-1}
            const int ct = k & 3, K = col_size(c, k), Kp = col_size(c, k - 1);
            const int Kn = (k + 1 < ncol) ? col_size(c, k + 1) : 0;
            load_col(c, k, s.kc, nullptr);
            load_col(c, k - 1, s.kp, nullptr);
            load_col(c, k + 1, s.kn, nullptr);
            __syncthreads();
            cx<R>* Pbar = Pb[pb];
            const cx<R>* Qn = Qb[qb];      // -A_bar_{k+1}
            // g_bar_k
            if (k > 0)
                dense_product<R, true>(Kp, K, KL, Pm, KL, Pbar, KL, T1, KL, s);
            const int ctn = (k + 1) & 3;
            for (int i = warp; i < K; i += NWARP) {
                int a0 = -1, a1 = -1, n0 = -1, n1 = -1;
                if (k > 0) col_src(ct, i, Kp, a0, a1);
                if (k + 1 < ncol) col_src_T(ctn, i, Kn, n0, n1);
                const bool ki = s.kc[i];
                for (int l = lane; l < K; l += 32) {
                    cx<R> v = czero<R>();
                    if (ki && s.kc[l]) {
                        if (k > 0) {
                            if (a0 >= 0 && s.kp[a0]) v = cadd(v, T1[(size_t)a0 * KL + l]);
                            if (a1 >= 0 && s.kp[a1]) v = cadd(v, T1[(size_t)a1 * KL + l]);
                            v = cscale(v, t);
                        } else {
                            v = Pbar[(size_t)i * KL + l];
                        }
                        if (k + 1 < ncol) {
                            int m0, m1;
                            col_src_T(ctn, l, Kn, m0, m1);
                            cx<R> w = czero<R>();
                            const bool kn0 = n0 >= 0 && s.kn[n0], kn1 = n1 >= 0 && s.kn[n1];
                            const bool km0 = m0 >= 0 && s.kn[m0], km1 = m1 >= 0 && s.kn[m1];
                            if (kn0 && km0) w = cadd(w, Qn[(size_t)n0 * KL + m0]);
                            if (kn0 && km1) w = cadd(w, Qn[(size_t)n0 * KL + m1]);
                            if (kn1 && km0) w = cadd(w, Qn[(size_t)n1 * KL + m0]);
                            if (kn1 && km1) w = cadd(w, Qn[(size_t)n1 * KL + m1]);
                            v = cadd(v, cscale(w, t2));     // - W A_bar W^T = + W Q W^T
                        }
                    }
                    gbar[(size_t)i * KL + l] = v;
                }
            }
            __syncthreads();
            // Q_k = g_k g_bar_k g_k  (= -A_bar_k)
            dense_product<R, false>(K, K, K, gbar, KL, gk, KL, T1, KL, s);
            cx<R>* Qk = Qb[qb ^ 1];
            dense_product<R, false>(K, K, K, gk, KL, T1, KL, Qk, KL, s);
            const int n = k >> 2;
            for (int i = threadIdx.x; i < K; i += NT)
                if (s.kc[i]) grad[(size_t)n * c.M + 4 * i + ct] = 2.0 * to_z(Qk[(size_t)i * KL + i]).re;
            // P_bar_{k-1} = P_bar_k g_k W_k^T
            if (k > 0) {
                dense_product<R, false>(KL, K, K, Pbar, KL, gk, KL, T1, KL, s);
                cx<R>* Pn = Pb[pb ^ 1];
                for (int r = warp; r < KL; r += NWARP)
                    for (int a = lane; a < Kp; a += 32) {
                        cx<R> v = czero<R>();
                        if (s.kp[a]) {
                            int b0, b1;
                            col_src_T(ct, a, K, b0, b1);
                            if (b0 >= 0 && s.kc[b0]) v = cadd(v, T1[(size_t)r * KL + b0]);
                            if (b1 >= 0 && s.kc[b1]) v = cadd(v, T1[(size_t)r * KL + b1]);
                            v = cscale(v, t);
                        }
                        Pn[(size_t)r * KL + a] = v;
                    }
                __syncthreads();
                pb ^= 1;
            }
            qb ^= 1;
        }
    }
    if constexpr (TC) {
        if (*(volatile int*)tst.ar.err() && threadIdx.x == 0 && status) status[ci] = ST_ETIMEOUT;
        tc::teardown(tst.ar);
    }
}

size_t grad_ws_elems(int N, int L, int seg_cols) {
    size_t KL = (size_t)col_KL(N);
    size_t ncol = 4 * (size_t)L;
    size_t nseg = (ncol + seg_cols - 1) / seg_cols;
    return (12 + 2 * nseg + 2 * ((size_t)seg_cols + 1)) * KL * KL;
}

cudaError_t launch_grad(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, const int* seg_cols, double* T, double* dT,
                        int32_t* status, cudaStream_t st) {
    if (nchains <= 0) return cudaSuccess;
    const bool tc = precision == 2;
    const size_t smem = sweep_smem_bytes(Kmax, tc);
    cudaError_t e;
    if (precision == 0) {
        e = cudaFuncSetAttribute(grad_kernel<double, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        grad_kernel<double, false><<<nchains, NT, smem, st>>>(
            chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status, leads,
            (zd*)ws, seg_cols, T, dT, status);
    } else if (tc) {
        e = cudaFuncSetAttribute(grad_kernel<df32, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        grad_kernel<df32, true><<<nchains, NT, smem, st>>>(
            chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status, leads,
            (zf*)ws, seg_cols, T, dT, status);
    } else {
        e = cudaFuncSetAttribute(grad_kernel<df32, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        grad_kernel<df32, false><<<nchains, NT, smem, st>>>(
            chains, order, nchains, Kmax, eta_device, (const zd*)leadout, lead_status, leads,
            (zf*)ws, seg_cols, T, dT, status);
    }
    return cudaGetLastError();
}

}  // namespace rgf
