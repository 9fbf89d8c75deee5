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
//
// Each chain runs on a cluster of C blocks (C SMs; C = 1, 2, 4 or 8, the
// largest with chains x C <= SMs).  Two schedules:
//   C = 2  pipeline: block 0 builds and inverts column k+1 while block 1
//          applies the strip product of column k; one cluster barrier per
//          column hands g_k over through a double buffer in L2.
//   else   team: every phase is shared -- the A_k build and the copy-out of
//          g_k by rows, the Gauss-Jordan panel redundantly (same data, same
//          result), its substitution and rank-b update by columns, the strip
//          product by columns; cluster barriers order the phases.
// With TC (precision RGF_MIXED_TC) the two dense contractions of a column
// step -- the Gauss-Jordan rank-b updates and the strip product -- run on the
// tcgen05 tensor cores by exact digit slicing of their double-float operands
// (rgf_tc.cuh); every block then holds the SM's TMEM for the whole launch.
#include <cooperative_groups.h>

#include "rgf_steps.cuh"

namespace rgf {

size_t sweep_smem_bytes(int Kmax, bool tc) {
    return sweep_total_bytes(Kmax, gj_panel_width(Kmax, tc), tc);
}

template <class R, bool TC>
__global__ void __launch_bounds__(NT, 1)
sweep_team_kernel(const ChainDev* __restrict__ chains, const int* __restrict__ order, int nchains,
             int Kmax, double eta_d, const zd* __restrict__ leadout,
             const int* __restrict__ lead_status, const LeadDev* __restrict__ leads,
             cx<R>* __restrict__ ws, double* __restrict__ Tout, int32_t* __restrict__ status) {
    namespace cg = cooperative_groups;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SweepSmem<R> s = carve<R>(smem_raw, Kmax, TC);
    cg::cluster_group cluster = cg::this_cluster();
    const Team tm{(int)cluster.block_rank(), (int)cluster.num_blocks()};
    const int ci = order[blockIdx.x / tm.C];
    const ChainDev ch = chains[ci];
    const int lst = lead_state(lead_status, ch.lead);
    if (lst != ST_OK) {            // every block of the cluster leaves here
        if (tm.rank == 0 && threadIdx.x == 0) { Tout[ci] = NAN; if (status) status[ci] = lst; }
        return;
    }
    const ChainCtx c = make_ctx(ch, leads[ch.lead], leadout, eta_d);
    const size_t B = (size_t)c.KL * c.KL;
    cx<R>* X = ws + ch.ws_off;
    cx<R>* G = X + B;
    cx<R>* P = X + 2 * B;
    cx<R>* Y = X + 3 * B;
    tc::State tst;
    if constexpr (TC) tc_attach<R>(Kmax, s, tst);
    int flag = 0;
    for (int k = 0; k < c.ncol; ++k) {
        load_col(c, k, s.kc, s.eps);
        load_col(c, k - 1, s.kp, nullptr);
        __syncthreads();
        flag |= inv_column<R>(c, k, G, G, X, s, tm);
        cl_sync(tm);               // g_k complete
        strip_column<R>(c, k, G, P, P, Y, s, tm);
        cl_sync(tm);               // P_k complete
    }
    if constexpr (TC) {
        if (*(volatile int*)tst.ar.err()) flag |= 4;
        tc::teardown(tst.ar);
    }
    if (tm.rank == 0) {
        const double T = trace_T<R>(c, P, X, G, Y, s);
        if (threadIdx.x == 0) {
            const int st = chain_status(c, flag, T);
            Tout[ci] = (st == ST_OK) ? T : NAN;
            if (status) status[ci] = st;
        }
    }
}

template <class R, bool TC>
__global__ void __launch_bounds__(NT, 1)
sweep_pipe_kernel(const ChainDev* __restrict__ chains, const int* __restrict__ order, int nchains,
                  int Kmax, double eta_d, const zd* __restrict__ leadout,
                  const int* __restrict__ lead_status, const LeadDev* __restrict__ leads,
                  cx<R>* __restrict__ ws, double* __restrict__ Tout, int32_t* __restrict__ status) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    SweepSmem<R> s = carve<R>(smem_raw, Kmax, TC);
    const int role = (int)cluster.block_rank();      // 0: inverse, 1: strip
    const int ci = order[blockIdx.x >> 1];
    const ChainDev ch = chains[ci];
    const int lst = lead_state(lead_status, ch.lead);
    if (lst != ST_OK) {            // both blocks of the cluster leave here
        if (role == 1 && threadIdx.x == 0) { Tout[ci] = NAN; if (status) status[ci] = lst; }
        return;
    }
    const ChainCtx c = make_ctx(ch, leads[ch.lead], leadout, eta_d);
    const size_t B = (size_t)c.KL * c.KL;
    cx<R>* X = ws + ch.ws_off;
    cx<R>* Gb[2] = {X + B, X + 2 * B};
    cx<R>* P = X + 3 * B;
    cx<R>* Y = X + 4 * B;
    int* flag_slot = reinterpret_cast<int*>(X + 5 * B);
    tc::State tst;
    if constexpr (TC) tc_attach<R>(Kmax, s, tst);
    if (role == 0) {
        int flag = 0;
        for (int k = 0; k < c.ncol; ++k) {
            load_col(c, k, s.kc, s.eps);
            load_col(c, k - 1, s.kp, nullptr);
            __syncthreads();
            flag |= inv_column<R>(c, k, Gb[(k + 1) & 1], Gb[k & 1], X, s);
            cluster.sync();        // g_k ready; block 1 is done with g_{k-1}
        }
        if constexpr (TC) {
            if (*(volatile int*)tst.ar.err()) flag |= 4;
            tc::teardown(tst.ar);
        }
        if (threadIdx.x == 0) *flag_slot = flag;
        cluster.sync();
    } else {
        for (int k = 0; k < c.ncol; ++k) {
            cluster.sync();
            load_col(c, k, s.kc, nullptr);
            load_col(c, k - 1, s.kp, nullptr);
            __syncthreads();
            strip_column<R>(c, k, Gb[k & 1], P, P, Y, s);
        }
        int tflag = 0;
        if constexpr (TC) {
            if (*(volatile int*)tst.ar.err()) tflag = 4;
            tc::teardown(tst.ar);
        }
        cluster.sync();
        const int flag = *(volatile int*)flag_slot | tflag;
        const double T = trace_T<R>(c, P, X, Gb[0], Y, s);
        if (threadIdx.x == 0) {
            const int st = chain_status(c, flag, T);
            Tout[ci] = (st == ST_OK) ? T : NAN;
            if (status) status[ci] = st;
        }
    }
}

template <class R, bool TC>
static cudaError_t launch_sweep_t(const ChainDev* chains, const int* order, int nchains, int Kmax,
                                  double eta_device, const zd* leadout, const int* lead_status,
                                  const LeadDev* leads, cx<R>* ws, double* T, int32_t* status,
                                  cudaStream_t st) {
    const size_t smem = sweep_smem_bytes(Kmax, TC);
    // Blocks per chain: the largest of 8, 4, 2, 1 with chains x C <= SMs.
    int dev = 0, nsm = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    int C = 8;
    while (C > 1 && (long long)nchains * C > nsm) C >>= 1;
    auto kern = (C == 2) ? sweep_pipe_kernel<R, TC> : sweep_team_kernel<R, TC>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * nchains, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, chains, order, nchains, Kmax, eta_device, leadout,
                              lead_status, leads, ws, T, status);
}

cudaError_t launch_sweep(int precision, const ChainDev* chains, const int* order, int nchains,
                         int Kmax, double eta_device, const void* leadout, const int* lead_status,
                         const LeadDev* leads, void* ws, double* T, int32_t* status,
                         cudaStream_t st) {
    if (nchains <= 0) return cudaSuccess;
    cudaError_t e;
    if (precision == 0)
        e = launch_sweep_t<double, false>(chains, order, nchains, Kmax, eta_device,
                                          (const zd*)leadout, lead_status, leads, (zd*)ws, T,
                                          status, st);
    else if (precision == 2)
        e = launch_sweep_t<df32, true>(chains, order, nchains, Kmax, eta_device,
                                       (const zd*)leadout, lead_status, leads, (zf*)ws, T, status,
                                       st);
    else
        e = launch_sweep_t<df32, false>(chains, order, nchains, Kmax, eta_device,
                                        (const zd*)leadout, lead_status, leads, (zf*)ws, T,
                                        status, st);
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace rgf
