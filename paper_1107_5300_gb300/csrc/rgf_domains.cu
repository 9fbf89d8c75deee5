// rgf_domains.cu -- the recursion of chains cut into more than two domains:
// the two lead-attached halves at the ends and ndom - 2 interior domains
// between them, every domain on its own SM at the same time; merge_body joins
// them (the method and the device bodies are in rgf_half.cuh).
#include "rgf_half.cuh"

namespace rgf {

// Block b runs domain b % ndom of chain order[b / ndom].
template <class R, bool TC>
__global__ void __launch_bounds__(NT, 1) domain_kernel(SweepArgs a, int bm) {
    const int ci = a.order[blockIdx.x / a.ndom], d = blockIdx.x % a.ndom;
    if (lead_state(a.lead_status, a.chains[ci].lead) != ST_OK) return;
    tc::State tst;
    if constexpr (TC) {
        SweepSmem<R> s = carve<R>(rgf_dyn_smem, a.Kmax, TC, bm);
        tc_attach<R>(a.Kmax, s, tst);
    }
    domain_body<R, TC>(a, ci, d, bm, &tst);
    if constexpr (TC) tc::teardown(tst.ar);
}

// Level `level` of the tree of joins of the interior domains: block b runs
// join b % njoin of chain order[b / njoin].  TCJ: the joins' products on the
// tensor cores (binary64 slicing).
template <class R, bool TCJ>
__global__ void __launch_bounds__(NT, 1) tree_kernel(SweepArgs a, int bm, int level, int njoin) {
    const int ci = a.order[blockIdx.x / njoin], j = blockIdx.x % njoin;
    if (lead_state(a.lead_status, a.chains[ci].lead) != ST_OK) return;
    tc::State tst;
    if constexpr (TCJ) {
        SweepSmem<double> s = carve<double>(rgf_dyn_smem, a.Kmax, true, bm);
        tc_attach<double>(a.Kmax, s, tst);
    }
    tree_join_body<R, TCJ>(a, ci, level, j, bm, &tst);
    if constexpr (TCJ) tc::teardown(tst.ar);
}

namespace {

auto domain_kern(int precision) {
    return precision == 0   ? domain_kernel<double, false>
           : precision == 3 ? domain_kernel<double, true>
           : precision == 2 ? domain_kernel<df32, true>
                            : domain_kernel<df32, false>;
}
// The joins: the tensor-core precisions on the tensor cores, binary64 sliced.
auto tree_kern(int precision) {
    return precision == 0   ? tree_kernel<double, false>
           : precision == 3 ? tree_kernel<double, true>
           : precision == 2 ? tree_kernel<df32, true>
                            : tree_kernel<df32, false>;
}
size_t tree_smem(int precision, int Kmax) {
    return uses_tc(precision) ? rec_smem(precision, Kmax) : f64_smem(precision, Kmax);
}

}  // namespace

cudaError_t configure_domains(int precision, int Kmax) {
    cudaError_t e = set_smem(domain_kern(precision), rec_smem(precision, Kmax));
    if (e != cudaSuccess) return e;
    return set_smem(tree_kern(precision), tree_smem(precision, Kmax));
}

cudaError_t launch_tree(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, int ndom, cudaStream_t st) {
    const int M = ndom - 2;
    if (nchains <= 0 || M < 2) return cudaSuccess;
    cudaError_t e = configure_domains(precision, Kmax);
    if (e != cudaSuccess) return e;
    const SweepArgs a = make_args(chains, order, nchains, Kmax, eta_device, leadout, lead_status,
                                  leads, ws, nullptr, nullptr, ndom);
    auto kern = tree_kern(precision);
    for (int level = 0; (1 << level) < M; ++level) {
        const int njoin = (M + (2 << level) - 1) / (2 << level);
        kern<<<nchains * njoin, NT, tree_smem(precision, Kmax), st>>>(a, launch_panel(precision, Kmax),
                                                                      level, njoin);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_domains(int precision, const ChainDev* chains, const int* order, int nchains,
                           int Kmax, double eta_device, const void* leadout,
                           const int* lead_status, const LeadDev* leads, void* ws, int ndom,
                           cudaStream_t st) {
    if (nchains <= 0) return cudaSuccess;
    cudaError_t e = configure_domains(precision, Kmax);
    if (e != cudaSuccess) return e;
    const SweepArgs a = make_args(chains, order, nchains, Kmax, eta_device, leadout, lead_status,
                                  leads, ws, nullptr, nullptr, ndom);
    domain_kern(precision)<<<nchains * ndom, NT, rec_smem(precision, Kmax), st>>>(
        a, launch_panel(precision, Kmax));
    return cudaGetLastError();
}

}  // namespace rgf
