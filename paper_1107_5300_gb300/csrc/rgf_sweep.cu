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
#include "rgf_steps.cuh"

namespace rgf {

size_t sweep_smem_bytes(int Kmax) {
    const int bm = gj_panel_width(Kmax);
    size_t b = 0;
    b += 2 * align16((size_t)Kmax * bm * 16);   // panel, pivot rows
    b += align16((size_t)bm * 16);              // rowbuf
    b += align16((size_t)Kmax * 16);            // colbuf
    b += align16(2 * 8 * 64 * 16);              // gemm tiles
    b += align16(16);                           // inv
    b += align16((size_t)Kmax * 8);             // eps
    b += align16(NWARP * 8);                    // red
    b += align16((size_t)Kmax * 4) * 2;         // perm, idx
    b += align16(16);                           // ctl
    b += align16((size_t)Kmax) * 3;             // kc, kp, kn
    return b;
}

template <class R>
__global__ void __launch_bounds__(NT, 1)
sweep_kernel(const ChainDev* __restrict__ chains, const int* __restrict__ order, int nchains,
             int Kmax, double eta_d, const zd* __restrict__ leadout,
             const int* __restrict__ lead_status, const LeadDev* __restrict__ leads,
             cx<R>* __restrict__ ws, double* __restrict__ Tout, int32_t* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SweepSmem<R> s = carve<R>(smem_raw, Kmax);
    const int ci = order[blockIdx.x];
    const ChainDev ch = chains[ci];
    const int lst = lead_state(lead_status, ch.lead);
    if (lst != ST_OK) {
        if (threadIdx.x == 0) { Tout[ci] = NAN; if (status) status[ci] = lst; }
        return;
    }
    const ChainCtx c = make_ctx(ch, leads[ch.lead], leadout, eta_d);
    const size_t B = (size_t)c.KL * c.KL;
    cx<R>* X = ws + ch.ws_off;
    cx<R>* G = X + B;
    cx<R>* P = G + B;
    cx<R>* Y = P + B;
    int flag = 0;
    for (int k = 0; k < c.ncol; ++k) {
        load_col(c, k, s.kc, s.eps);
        load_col(c, k - 1, s.kp, nullptr);
        __syncthreads();
        flag |= fwd_column<R>(c, k, G, G, P, P, X, Y, s);
    }
    const double T = trace_T<R>(c, P, X, G, Y, s);
    if (threadIdx.x == 0) {
        const int st = chain_status(c, flag, T);
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
