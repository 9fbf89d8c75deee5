// rgf_sweep.cu -- the forward RGF sweep (Eqs. 4-5) and the Landauer trace
// (Eq. 2), one thread block per chain (ribbon, energy).
//
// The paper slices the ribbon into cross-sections and applies, slice after
// slice, g_j = (z - H_jj - V^T g_{j-1} V)^-1 together with the corner block
// G_1j = G_1,j-1 V g_j (Eqs. 4-5).  Here each unit cell (2N orbitals) is
// sliced further into its four atom columns (x = 0, a, 1.5a, 2.5a): a column
// has no internal hopping, neighbouring columns are coupled by t*I (same row)
// or by a bidiagonal t-stencil (rows j +- 1).  The recursion is the same
// Dyson step on blocks of KL = ceil(N/2) or KR = floor(N/2) orbitals, 4L steps
// per chain, and reaches the same G_1L:
//
//   A_k   = (z - eps_k) I - t^2 S_k^T g_{k-1} S_k   (- Sigma_L at k = 0,
//                                                   - Sigma_R at k = 4L-1)
//   g_k   = A_k^-1                                  (Gauss-Jordan, pivoted)
//   P_k   = (P_{k-1} W_k) g_k,   P_0 = g_0          (P_k = G_{first col, k})
//   T     = Tr[Gamma_L P Gamma_R P^dagger]          (binary64)
//
// S_k is the 1- or 2-point source stencil of the column coupling; the product
// V^T g V is a gather-and-contract over at most 4 entries of g_{k-1} per entry.
// Removed atoms become identity rows/columns with zero couplings (an exact
// equivalence to dropping them).
#include "rgf_device.cuh"
#include "rgf_internal.h"

namespace rgf {

template <class R>
struct SweepSmem {
    GJSmem<R> gj;
    cx<R>* gemm;
    uint8_t* kc;
    uint8_t* kp;
    double* eps;
    double* red;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

size_t sweep_smem_bytes(int Kmax) {
    size_t b = 0;
    b += 3 * align16((size_t)Kmax * 16);   // rowbuf, colbuf, colval
    b += align16(2 * 8 * 64 * 16);         // gemm tiles
    b += align16(16);                      // inv
    b += align16((size_t)Kmax * 8) * 2;    // colabs, eps
    b += align16(NWARP * 8);               // red
    b += align16((size_t)Kmax * 4) * 2;    // perm, idx
    b += align16(16);                      // ctl
    b += align16((size_t)Kmax) * 2;        // kc, kp
    return b;
}

template <class R>
__device__ SweepSmem<R> carve(unsigned char* base, int Kmax) {
    SweepSmem<R> s;
    size_t o = 0;
    auto take = [&](size_t bytes) { unsigned char* p = base + o; o += align16(bytes); return p; };
    s.gj.rowbuf = (cx<R>*)take((size_t)Kmax * 16);
    s.gj.colbuf = (cx<R>*)take((size_t)Kmax * 16);
    s.gj.colval = (cx<R>*)take((size_t)Kmax * 16);
    s.gemm = (cx<R>*)take(2 * 8 * 64 * 16);
    s.gj.inv = (zd*)take(16);
    s.gj.colabs = (double*)take((size_t)Kmax * 8);
    s.eps = (double*)take((size_t)Kmax * 8);
    s.red = (double*)take(NWARP * 8);
    s.gj.perm = (int*)take((size_t)Kmax * 4);
    s.gj.idx = (int*)take((size_t)Kmax * 4);
    s.gj.ctl = (int*)take(16);
    s.kc = (uint8_t*)take((size_t)Kmax);
    s.kp = (uint8_t*)take((size_t)Kmax);
    return s;
}

// Source stencil of the coupling into column type c: entry i of column c is
// bonded to entries a0, a1 (-1 = none) of the previous column (size Kp).
__device__ __forceinline__ void col_src(int c, int i, int Kp, int& a0, int& a1) {
    if (c == 1 || c == 3) { a0 = i; a1 = -1; }
    else if (c == 2) { a0 = i; a1 = (i + 1 < Kp) ? i + 1 : -1; }
    else { a0 = i - 1; a1 = (i < Kp) ? i : -1; }
}

template <class R>
__device__ __forceinline__ cx<R> ld_z(const zd* p) { return from_z<R>(p->re, p->im); }

// Tr[Gamma_L P Gamma_R P^dagger] in binary64.  Pz: KL x KR (ld KL), Gamma_L
// KL x KL, Gamma_R KR x KR.  Uses Xs, Zs (KL x KL zd each) as scratch.
__device__ double trace_T(const zd* Pz, int KL, int KR, const zd* GamL, const zd* GamR, zd* Xs,
                          zd* Zs, zd* gsm, double* red) {
    cta_gemm<double, false, false>(KL, KR, KL, GamL, KL, Pz, KL, Xs, KL, GEMM_SET, gsm);
    cta_gemm<double, false, false>(KL, KR, KR, Pz, KL, GamR, KR, Zs, KL, GEMM_SET, gsm);
    double acc = 0.0;
    for (int e = threadIdx.x; e < KL * KR; e += NT) {
        int a = e / KR, b = e % KR;
        zd x = Xs[(size_t)a * KL + b], zz = Zs[(size_t)a * KL + b];
        acc += x.re * zz.re + x.im * zz.im;    // Re(x * conj(z))
    }
    return block_sum(acc, red);
}

template <class R>
__global__ void __launch_bounds__(NT, 1)
sweep_kernel(const ChainDev* __restrict__ chains, const int* __restrict__ order, int nchains,
             int Kmax, double eta_d, const zd* __restrict__ leadout,
             const int* __restrict__ lead_status, const LeadDev* __restrict__ leads,
             cx<R>* __restrict__ ws, double* __restrict__ Tout, int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepSmem<R> s = carve<R>(smem_raw, Kmax);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int ci = order[blockIdx.x];
    const ChainDev ch = chains[ci];
    int lst = lead_status[2 * ch.lead];
    if (lst == ST_OK) lst = lead_status[2 * ch.lead + 1];
    if (lst != ST_OK) {
        if (tid == 0) { Tout[ci] = NAN; if (status) status[ci] = lst; }
        return;
    }
    const LeadDev ldv = leads[ch.lead];
    const int N = ch.N, L = ch.L, M = 2 * N, KL = col_KL(N), KR = col_KR(N);
    const zd* SigL = leadout + ldv.off;
    const zd* SigR = SigL + (size_t)KL * KL;
    const zd* GamL = SigR + (size_t)KR * KR;
    const zd* GamR = GamL + (size_t)KL * KL;
    cx<R>* X = ws + ch.ws_off;
    cx<R>* G = X + (size_t)KL * KL;
    cx<R>* P = G + (size_t)KL * KL;
    cx<R>* Y = P + (size_t)KL * KL;
    const double t = ch.t, t2 = t * t;
    const zd z = {ch.E, eta_d};
    int flag = 0;
    const int ncol = 4 * L;
    for (int k = 0; k < ncol; ++k) {
        const int n = k >> 2, c = k & 3;
        const int K = (c < 2) ? KL : KR;
        const int cp = (c + 3) & 3;
        const int Kp = (cp < 2) ? KL : KR;
        const int np = (c == 0) ? n - 1 : n;
        for (int i = tid; i < K; i += NT) {
            size_t o = (size_t)n * M + 4 * i + c;
            s.kc[i] = ch.rem ? (ch.rem[o] == 0) : 1;
            s.eps[i] = ch.eps[o];
        }
        if (k > 0)
            for (int i = tid; i < Kp; i += NT) {
                size_t o = (size_t)np * M + 4 * i + cp;
                s.kp[i] = ch.rem ? (ch.rem[o] == 0) : 1;
            }
        __syncthreads();
        // Strip input Y = P_{k-1} W_k (KL x K): sparse, two taps per column.
        if (k > 0) {
            for (int r = warp; r < KL; r += NWARP)
                for (int l = lane; l < K; l += 32) {
                    cx<R> v = czero<R>();
                    if (s.kc[l]) {
                        int a0, a1;
                        col_src(c, l, Kp, a0, a1);
                        if (a0 >= 0 && s.kp[a0]) v = cadd(v, P[(size_t)r * KL + a0]);
                        if (a1 >= 0 && s.kp[a1]) v = cadd(v, P[(size_t)r * KL + a1]);
                        v = cscale(v, t);
                    }
                    Y[(size_t)r * KL + l] = v;
                }
        }
        // A_k into X: diagonal part minus the gathered-and-contracted Sigma_k.
        for (int i = warp; i < K; i += NWARP) {
            int a0 = -1, a1 = -1;
            if (k > 0) col_src(c, i, Kp, a0, a1);
            const bool ki = s.kc[i];
            for (int l = lane; l < K; l += 32) {
                cx<R> v;
                if (!ki || !s.kc[l]) {
                    v = (i == l) ? from_z<R>(1.0, 0.0) : czero<R>();
                } else {
                    cx<R> sig = czero<R>();
                    if (k == 0) {
                        sig = ld_z<R>(SigL + (size_t)i * KL + l);
                    } else {
                        int b0, b1;
                        col_src(c, l, Kp, b0, b1);
                        const bool ka0 = a0 >= 0 && s.kp[a0], ka1 = a1 >= 0 && s.kp[a1];
                        const bool kb0 = b0 >= 0 && s.kp[b0], kb1 = b1 >= 0 && s.kp[b1];
                        if (ka0 && kb0) sig = cadd(sig, G[(size_t)a0 * KL + b0]);
                        if (ka0 && kb1) sig = cadd(sig, G[(size_t)a0 * KL + b1]);
                        if (ka1 && kb0) sig = cadd(sig, G[(size_t)a1 * KL + b0]);
                        if (ka1 && kb1) sig = cadd(sig, G[(size_t)a1 * KL + b1]);
                        sig = cscale(sig, t2);
                    }
                    if (k == ncol - 1) sig = cadd(sig, ld_z<R>(SigR + (size_t)i * KR + l));
                    v = (i == l) ? from_z<R>(z.re - s.eps[i], z.im) : czero<R>();
                    v = csub(v, sig);
                }
                X[(size_t)i * KL + l] = v;
            }
        }
        __syncthreads();
        flag |= cta_gj_invert<R>(X, K, KL, G, KL, s.gj);
        if (k == 0) {
            for (int i = warp; i < K; i += NWARP)
                for (int l = lane; l < K; l += 32) P[(size_t)i * KL + l] = G[(size_t)i * KL + l];
            __syncthreads();
        } else {
            cta_gemm<R, false, false>(KL, K, K, Y, KL, G, KL, P, KL, GEMM_SET, s.gemm);
        }
    }
    // Eq. 2 in binary64.
    const zd* Pz;
    if (sizeof(R) == sizeof(double)) {
        Pz = reinterpret_cast<const zd*>(P);
    } else {
        zd* Xz = reinterpret_cast<zd*>(X);
        for (int i = warp; i < KL; i += NWARP)
            for (int l = lane; l < KR; l += 32) Xz[(size_t)i * KL + l] = to_z(P[(size_t)i * KL + l]);
        __syncthreads();
        Pz = Xz;
    }
    double T = trace_T(Pz, KL, KR, GamL, GamR, reinterpret_cast<zd*>(G), reinterpret_cast<zd*>(Y),
                       reinterpret_cast<zd*>(s.gemm), s.red);
    if (tid == 0) {
        int st = ST_OK;
        if (flag & 1) st = ST_ESINGULAR;
        else if ((flag & 2) || !isfinite(T)) st = ST_ENONFINITE;
        Tout[ci] = (st == ST_OK) ? T : NAN;
        if (status) status[ci] = st;
    }
}

cudaError_t launch_sweep(int precision, const ChainDev* chains, const int* order, int nchains,
                         int Kmax, double eta_device, const void* leadout, const int* lead_status,
                         const LeadDev* leads, void* ws, double* T, int32_t* status,
                         cudaStream_t st) {
    if (nchains <= 0) return cudaSuccess;
    size_t smem = sweep_smem_bytes(Kmax);
    cudaError_t e;
    if (precision == 0) {
        e = cudaFuncSetAttribute(sweep_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        sweep_kernel<double><<<nchains, NT, smem, st>>>(chains, order, nchains, Kmax, eta_device,
                                                       (const zd*)leadout, lead_status, leads,
                                                       (zd*)ws, T, status);
    } else {
        e = cudaFuncSetAttribute(sweep_kernel<df32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        if (e != cudaSuccess) return e;
        sweep_kernel<df32><<<nchains, NT, smem, st>>>(chains, order, nchains, Kmax, eta_device,
                                                     (const zd*)leadout, lead_status, leads,
                                                     (zf*)ws, T, status);
    }
    return cudaGetLastError();
}

}  // namespace rgf
