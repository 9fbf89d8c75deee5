// rgf_sweep.cu -- the three-launch schedule of the forward sweep: end-column
// preparation, half sweeps and joins as separate launches over every chain
// (the method and the device bodies are in rgf_half.cuh).
#include "rgf_half.cuh"

namespace rgf {

size_t sweep_smem_bytes(int Kmax, bool tc) {
    return sweep_total_bytes(Kmax, gj_panel_width(Kmax, tc), tc);
}

bool tc_layout_fits(int Kmax) {
    return sweep_total_bytes(Kmax, gj_panel_width(Kmax, true), true) <= 232448;
}

// Three-launch schedule: each kernel runs one step for every half (or chain),
// blocks in the order of `order`.
template <class R>
__global__ void __launch_bounds__(NT, 1) prep_kernel(SweepArgs a, int bm) {
    const int ci = a.order[blockIdx.x >> 1], h = blockIdx.x & 1;
    if (lead_state(a.lead_status, a.chains[ci].lead) != ST_OK) return;     // reported by the merge
    prep_body<R>(a, ci, h, bm);
}

template <class R, bool TC>
__global__ void __launch_bounds__(NT, 1) half_kernel(SweepArgs a, int bm) {
    const int ci = a.order[blockIdx.x >> 1], h = blockIdx.x & 1;
    if (lead_state(a.lead_status, a.chains[ci].lead) != ST_OK) return;
    tc::State tst;
    if constexpr (TC) {
        SweepSmem<R> s = carve<R>(rgf_dyn_smem, a.Kmax, TC, bm);
        tc_attach<R>(a.Kmax, s, tst);
    }
    half_body<R, TC>(a, ci, h, bm, &tst);
    if constexpr (TC) tc::teardown(tst.ar);
}

template <class R>
__global__ void __launch_bounds__(NT, 1) merge_kernel(SweepArgs a, int bm) {
    merge_body<R>(a, a.order[blockIdx.x], bm);
}

// The joins of chains cut into more than two domains in a tensor-core
// precision: products on the tensor cores (binary64 slicing).
template <class R>
__global__ void __launch_bounds__(NT, 1) merge_tc_kernel(SweepArgs a, int bm) {
    tc::State tst;
    SweepSmem<double> s = carve<double>(rgf_dyn_smem, a.Kmax, true, bm);
    tc_attach<double>(a.Kmax, s, tst);
    merge_body<R, true>(a, a.order[blockIdx.x], bm, &tst);
    tc::teardown(tst.ar);
}

namespace {

// The shared-memory limits of the three-launch kernels of `precision`.
cudaError_t configure_phased(int precision, int Kmax) {
    const size_t f64 = f64_smem(precision, Kmax), rec = rec_smem(precision, Kmax);
    cudaError_t e;
    if (binary64(precision)) {
        if ((e = set_smem(prep_kernel<double>, f64)) != cudaSuccess) return e;
        if ((e = set_smem(merge_kernel<double>, f64)) != cudaSuccess) return e;
        return set_smem(precision == 3 ? half_kernel<double, true> : half_kernel<double, false>, rec);
    }
    if ((e = set_smem(prep_kernel<df32>, f64)) != cudaSuccess) return e;
    if ((e = set_smem(merge_kernel<df32>, f64)) != cudaSuccess) return e;
    return set_smem(precision == 2 ? half_kernel<df32, true> : half_kernel<df32, false>, rec);
}

}  // namespace

cudaError_t configure_sweep(int precision, int Kmax) {
    cudaError_t e = configure_phased(precision, Kmax);
    if (e == cudaSuccess) e = configure_batch(precision, Kmax);
    return e == cudaSuccess ? configure_domains(precision, Kmax) : e;
}

cudaError_t launch_prep(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, cudaStream_t st, int ndom) {
    if (nchains <= 0) return cudaSuccess;
    cudaError_t e = configure_phased(precision, Kmax);
    if (e != cudaSuccess) return e;
    const SweepArgs a = make_args(chains, order, nchains, Kmax, eta_device, leadout, lead_status,
                                  leads, ws, nullptr, nullptr, ndom);
    auto kern = binary64(precision) ? prep_kernel<double> : prep_kernel<df32>;
    kern<<<2 * nchains, NT, f64_smem(precision, Kmax), st>>>(a, launch_panel(precision, Kmax));
    return cudaGetLastError();
}

cudaError_t launch_half(int precision, const ChainDev* chains, const int* order, int nchains,
                        int Kmax, double eta_device, const void* leadout, const int* lead_status,
                        const LeadDev* leads, void* ws, cudaStream_t st, int ndom) {
    if (nchains <= 0) return cudaSuccess;
    if (ndom > 2)
        return launch_domains(precision, chains, order, nchains, Kmax, eta_device, leadout,
                              lead_status, leads, ws, ndom, st);
    cudaError_t e = configure_phased(precision, Kmax);
    if (e != cudaSuccess) return e;
    const SweepArgs a = make_args(chains, order, nchains, Kmax, eta_device, leadout, lead_status,
                                  leads, ws, nullptr, nullptr);
    auto kern = precision == 0   ? half_kernel<double, false>
                : precision == 3 ? half_kernel<double, true>
                : precision == 2 ? half_kernel<df32, true>
                                 : half_kernel<df32, false>;
    kern<<<2 * nchains, NT, rec_smem(precision, Kmax), st>>>(a, launch_panel(precision, Kmax));
    return cudaGetLastError();
}

cudaError_t launch_merge(int precision, const ChainDev* chains, const int* order, int nchains,
                         int Kmax, double eta_device, const void* leadout, const int* lead_status,
                         const LeadDev* leads, void* ws, double* T, int32_t* status,
                         cudaStream_t st, int ndom) {
    if (nchains <= 0) return cudaSuccess;
    cudaError_t e = configure_phased(precision, Kmax);
    if (e != cudaSuccess) return e;
    if (ndom > 3) {
        e = launch_tree(precision, chains, order, nchains, Kmax, eta_device, leadout, lead_status,
                        leads, ws, ndom, st);
        if (e != cudaSuccess) return e;
    }
    const SweepArgs a = make_args(chains, order, nchains, Kmax, eta_device, leadout, lead_status,
                                  leads, ws, T, status, ndom);
    if (ndom > 2 && uses_tc(precision)) {
        auto kern = binary64(precision) ? merge_tc_kernel<double> : merge_tc_kernel<df32>;
        const size_t smem = rec_smem(precision, Kmax);
        if ((e = set_smem(kern, smem)) != cudaSuccess) return e;
        kern<<<nchains, NT, smem, st>>>(a, launch_panel(precision, Kmax));
        return cudaGetLastError();
    }
    auto kern = binary64(precision) ? merge_kernel<double> : merge_kernel<df32>;
    kern<<<nchains, NT, f64_smem(precision, Kmax), st>>>(a, launch_panel(precision, Kmax));
    return cudaGetLastError();
}

}  // namespace rgf
