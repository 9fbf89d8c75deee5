// rgf_api.cu -- host side of the C ABI declared in include/rgf.h: ribbon
// instances, argument checks, workspace, launch order, status reporting.
//
// Call flow of rgf_conductance (the paper's step list: input and defects ->
// lead self-energies -> recursion on the device -> conductance):
//   1. one lead problem per chain (pristine ribbon of the chain's width at the
//      chain's energy), decimated on the device (rgf_lead.cu);
//   2. the column-sliced recursion as two halves per chain, one from each
//      lead, joined by one Dyson step, and the trace (rgf_sweep.cu: end-column
//      preparation, half sweeps, merge); chains are launched longest first so
//      that the hardware block scheduler balances uneven chains across SMs;
//   3. T and the per-chain status words return to the host.
// Only on-site energies / masks (at ribbon build), energies and T cross the
// host-device boundary.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "rgf.h"
#include "rgf_internal.h"

struct rgf_ribbon {
    int N, L;
    double t;
    double* eps;      // device [L*2N]
    uint8_t* rem;     // device [L*2N] or nullptr
    int device;
};

namespace {

thread_local std::string g_last_error;

// Events around the phases of the last call: [0] lead decimation [1]
// end-column preparation [2] half sweeps (or the gradient sweep) [3] merge [4].
constexpr int kProfEvents = 5;
struct Profile {
    bool on = false, recorded = false;
    cudaEvent_t ev[kProfEvents] = {};
};
Profile g_prof;

cudaError_t prof_record(int i, cudaStream_t st) {
    if (!g_prof.on) return cudaSuccess;
    if (!g_prof.ev[i]) {
        cudaError_t e = cudaEventCreate(&g_prof.ev[i]);
        if (e != cudaSuccess) return e;
    }
    return cudaEventRecord(g_prof.ev[i], st);
}

rgf_status fail(rgf_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

rgf_status cuda_fail(cudaError_t e, const char* what) {
    return fail(RGF_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define RGF_CUDA(call, what)                       \
    do {                                           \
        cudaError_t _e = (call);                   \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

// SplitMix64 (Steele, Lea, Flood 2014) as a counter-based generator.
inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
inline double uniform01(uint64_t seed, uint64_t i) {
    uint64_t bits = mix64(seed + (i + 1) * 0x9E3779B97F4A7C15ull);
    return (double)(bits >> 11) * 0x1.0p-53;
}

rgf_status check_desc(const rgf_ribbon_desc* d) {
    if (!d) return fail(RGF_EINVAL, "desc is NULL");
    if (d->N < 2 || d->N > 2047) return fail(RGF_EINVAL, "N must be in [2, 2047]");
    if (d->L < 1) return fail(RGF_EINVAL, "L must be >= 1");
    if (!std::isfinite(d->t) || d->t == 0.0) return fail(RGF_EINVAL, "t must be finite and nonzero");
    if (!d->onsite && !(d->anderson_W >= 0.0 && std::isfinite(d->anderson_W)))
        return fail(RGF_EINVAL, "anderson_W must be finite and >= 0");
    if (!d->removed && !(d->edge_p >= 0.0 && d->edge_p <= 1.0))
        return fail(RGF_EINVAL, "edge_p must be in [0, 1]");
    return RGF_OK;
}

struct DevBuf {
    void* p = nullptr;
    cudaStream_t st = nullptr;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, st);
    }
    cudaError_t alloc(size_t bytes, cudaStream_t s) {
        st = s;
        return cudaMallocAsync(&p, bytes ? bytes : 16, s);
    }
};

struct Plan {
    std::vector<rgf::ChainDev> chains;
    std::vector<rgf::LeadDev> leads;
    std::vector<int> order;
    std::vector<int> seg_cols;
    size_t ws_elems = 0, lead_ws_elems = 0, lead_out_elems = 0, grad_elems = 0;
    int Kmax = 1;
};

// grad: size the gradient workspace with checkpoints every ckpt_stride cells
// (<= 0: ceil(sqrt(L))).
rgf_status make_plan(const rgf_ribbon* const* rib, int nchains, Plan& pl, bool grad = false,
                     int ckpt_stride = 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    pl.chains.resize(nchains);
    pl.leads.resize(nchains);
    pl.seg_cols.resize(nchains);
    std::vector<double> cost(nchains);
    for (int c = 0; c < nchains; ++c) {
        const rgf_ribbon* r = rib[c];
        if (!r) return fail(RGF_EINVAL, "rib[" + std::to_string(c) + "] is NULL");
        if (r->device != dev) return fail(RGF_EINVAL, "ribbon was built on another device");
        rgf::ChainDev& ch = pl.chains[c];
        ch.eps = r->eps;
        ch.rem = r->rem;
        ch.N = r->N;
        ch.L = r->L;
        ch.t = r->t;
        ch.E = 0.0;   // filled on the device from the energy array
        ch.lead = c;
        ch.ws_off = pl.ws_elems;
        ch.grad_off = pl.grad_elems;
        if (grad) {
            int stride = ckpt_stride > 0 ? std::min(ckpt_stride, r->L)
                                         : std::max(1, (int)std::ceil(std::sqrt((double)r->L)));
            pl.seg_cols[c] = 4 * stride;
            pl.ws_elems += rgf::grad_ws_elems(r->N, r->L, pl.seg_cols[c]);
            pl.grad_elems += (size_t)r->L * 2 * r->N;
        } else {
            pl.seg_cols[c] = 0;
            pl.ws_elems += rgf::sweep_ws_elems(r->N);
        }
        rgf::LeadDev& ld = pl.leads[c];
        ld.N = r->N;
        ld.t = r->t;
        ld.E = 0.0;
        ld.off = pl.lead_out_elems;
        pl.lead_out_elems += rgf::lead_out_elems(r->N);
        ld.ws_off = pl.lead_ws_elems;
        pl.lead_ws_elems += rgf::lead_ws_elems(r->N);
        pl.Kmax = std::max(pl.Kmax, rgf::col_KL(r->N));
        double KL = rgf::col_KL(r->N);
        cost[c] = KL * KL * KL * (double)r->L;
    }
    pl.order.resize(nchains);
    for (int c = 0; c < nchains; ++c) pl.order[c] = c;
    std::stable_sort(pl.order.begin(), pl.order.end(),
                     [&](int a, int b) { return cost[a] > cost[b]; });
    return RGF_OK;
}

// Energies into the descriptors.  A non-finite energy reaches the lead
// kernel, which reports its chain as RGF_EINVAL.
__global__ void fill_energy(rgf::ChainDev* chains, rgf::LeadDev* leads, const double* E, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        double e = E[i];
        chains[i].E = e;
        leads[i].E = e;
    }
}

// Runs the whole path on `st`: lead decimation, then the forward sweep (or,
// with dT_dev, the checkpointed two-sided gradient sweep).  E_dev, T_dev, status_dev,
// dT_dev: device.
rgf_status run_path(const rgf_ribbon* const* rib, const double* E_dev, int nchains,
                    double eta_device, double eta_lead, int precision, cudaStream_t st,
                    double* T_dev, int32_t* status_dev, double* dT_dev = nullptr,
                    int ckpt_stride = 0, int out_mode = rgf::OUT_GRAD) {
    if (nchains < 0) return fail(RGF_EINVAL, "nchains < 0");
    if (nchains == 0) return RGF_OK;
    if (!rib || !E_dev || !T_dev) return fail(RGF_EINVAL, "NULL argument");
    if (precision != RGF_FP64 && precision != RGF_MIXED && precision != RGF_MIXED_TC)
        return fail(RGF_EINVAL, "unknown precision");
    if (!(eta_device >= 0.0) || !(eta_lead > 0.0) || !std::isfinite(eta_device) ||
        !std::isfinite(eta_lead))
        return fail(RGF_EINVAL, "eta_device must be >= 0 and eta_lead > 0 (finite)");
    const bool grad = dT_dev != nullptr;
    Plan pl;
    rgf_status s = make_plan(rib, nchains, pl, grad, ckpt_stride);
    if (s != RGF_OK) return s;

    const size_t nC = pl.chains.size() * sizeof(rgf::ChainDev);
    const size_t nL = pl.leads.size() * sizeof(rgf::LeadDev);
    const size_t nO = pl.order.size() * sizeof(int);
    std::vector<unsigned char> hdr(nC + nL + 2 * nO);
    std::memcpy(hdr.data(), pl.chains.data(), nC);
    std::memcpy(hdr.data() + nC, pl.leads.data(), nL);
    std::memcpy(hdr.data() + nC + nL, pl.order.data(), nO);
    std::memcpy(hdr.data() + nC + nL + nO, pl.seg_cols.data(), nO);

    DevBuf dhdr, dws, dlws, dlout, dlst;
    RGF_CUDA(dhdr.alloc(hdr.size(), st), "cudaMallocAsync(descriptors)");
    cudaError_t ae = dws.alloc(pl.ws_elems * 16, st);
    if (ae == cudaErrorMemoryAllocation) return fail(RGF_ENOMEM, "workspace allocation failed");
    RGF_CUDA(ae, "cudaMallocAsync(workspace)");
    RGF_CUDA(dlws.alloc(pl.lead_ws_elems * 16, st), "cudaMallocAsync(lead workspace)");
    RGF_CUDA(dlout.alloc(pl.lead_out_elems * 16, st), "cudaMallocAsync(lead output)");
    RGF_CUDA(dlst.alloc(2 * sizeof(int) * nchains, st), "cudaMallocAsync(lead status)");
    RGF_CUDA(cudaMemcpyAsync(dhdr.p, hdr.data(), hdr.size(), cudaMemcpyHostToDevice, st),
             "cudaMemcpyAsync(descriptors)");
    if (grad) RGF_CUDA(cudaMemsetAsync(dT_dev, 0, pl.grad_elems * sizeof(double), st), "cudaMemsetAsync");
    double* dgrad = (out_mode & rgf::OUT_GRAD) ? dT_dev : nullptr;
    double* drho = (out_mode & rgf::OUT_LDOS) ? dT_dev : nullptr;
    auto* dchains = (rgf::ChainDev*)dhdr.p;
    auto* dleads = (rgf::LeadDev*)((unsigned char*)dhdr.p + nC);
    auto* dorder = (int*)((unsigned char*)dhdr.p + nC + nL);
    auto* dseg = (int*)((unsigned char*)dhdr.p + nC + nL + nO);
    fill_energy<<<(nchains + 255) / 256, 256, 0, st>>>(dchains, dleads, E_dev, nchains);
    RGF_CUDA(cudaGetLastError(), "fill_energy launch");
    RGF_CUDA(prof_record(0, st), "cudaEventRecord");
    RGF_CUDA(rgf::launch_lead(dleads, nchains, pl.Kmax, eta_lead, dlws.p, dlout.p, (int*)dlst.p,
                              nullptr, st),
             "lead decimation launch");
    RGF_CUDA(prof_record(1, st), "cudaEventRecord");
    if (grad) {
        RGF_CUDA(prof_record(2, st), "cudaEventRecord");
        RGF_CUDA(rgf::launch_grad(precision, dchains, dorder, nchains, pl.Kmax, eta_device,
                                  dlout.p, (int*)dlst.p, dleads, dws.p, dseg, T_dev, dgrad, drho,
                                  out_mode, status_dev, st),
                 "gradient sweep launch");
        RGF_CUDA(prof_record(3, st), "cudaEventRecord");
    } else {
        RGF_CUDA(rgf::launch_prep(precision, dchains, dorder, nchains, pl.Kmax, eta_device,
                                  dlout.p, (int*)dlst.p, dleads, dws.p, st),
                 "end-column preparation launch");
        RGF_CUDA(prof_record(2, st), "cudaEventRecord");
        RGF_CUDA(rgf::launch_half(precision, dchains, dorder, nchains, pl.Kmax, eta_device,
                                  dlout.p, (int*)dlst.p, dleads, dws.p, st),
                 "half sweep launch");
        RGF_CUDA(prof_record(3, st), "cudaEventRecord");
        RGF_CUDA(rgf::launch_merge(precision, dchains, dorder, nchains, pl.Kmax, eta_device,
                                   dlout.p, (int*)dlst.p, dleads, dws.p, T_dev, status_dev, st),
                 "merge launch");
    }
    RGF_CUDA(prof_record(4, st), "cudaEventRecord");
    if (g_prof.on) g_prof.recorded = true;
    return RGF_OK;
}

// out[i] = sum_c w[c] g[c * n + i]: the weighted sum over chains of per-chain
// gradients (one thread per site, chains summed in order: deterministic).
__global__ void weighted_chain_sum(const double* __restrict__ g, const double* __restrict__ w,
                                   int nchains, size_t n, double* __restrict__ out) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double acc = 0.0;
    for (int c = 0; c < nchains; ++c) acc = fma(w[c], g[(size_t)c * n + i], acc);
    out[i] = acc;
}

// Host-buffer front end of run_path: copies E in and T (and dT) out on the
// legacy default stream, synchronises, returns the first per-chain failure.
rgf_status run_host(const rgf_ribbon* const* rib, const double* E, int nchains, double eta_device,
                    double eta_lead, int precision, double* T, int32_t* chain_status,
                    double* dT = nullptr, int ckpt_stride = 0, int out_mode = rgf::OUT_GRAD) {
    if (nchains < 0 || (nchains > 0 && (!rib || !E || !T)))
        return fail(RGF_EINVAL, "NULL argument or nchains < 0");
    if (nchains == 0) return RGF_OK;
    for (int i = 0; i < nchains; ++i) {
        if (!std::isfinite(E[i])) return fail(RGF_EINVAL, "non-finite energy");
        if (!rib[i]) return fail(RGF_EINVAL, "NULL ribbon");
    }
    size_t ng = 0;
    if (dT)
        for (int i = 0; i < nchains; ++i) ng += (size_t)rib[i]->L * 2 * rib[i]->N;
    cudaStream_t st = 0;
    std::vector<double> hT(nchains);
    std::vector<int32_t> hs(nchains);
    {
        DevBuf dE, dTt, dS, dG;
        RGF_CUDA(dE.alloc(nchains * sizeof(double), st), "cudaMallocAsync");
        RGF_CUDA(dTt.alloc(nchains * sizeof(double), st), "cudaMallocAsync");
        RGF_CUDA(dS.alloc(nchains * sizeof(int32_t), st), "cudaMallocAsync");
        if (dT) RGF_CUDA(dG.alloc(ng * sizeof(double), st), "cudaMallocAsync");
        RGF_CUDA(cudaMemcpyAsync(dE.p, E, nchains * sizeof(double), cudaMemcpyHostToDevice, st), "H2D");
        rgf_status s = run_path(rib, (const double*)dE.p, nchains, eta_device, eta_lead, precision,
                                st, (double*)dTt.p, (int32_t*)dS.p, (double*)dG.p, ckpt_stride,
                                out_mode);
        if (s != RGF_OK) return s;
        RGF_CUDA(cudaMemcpyAsync(hT.data(), dTt.p, nchains * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H");
        RGF_CUDA(cudaMemcpyAsync(hs.data(), dS.p, nchains * sizeof(int32_t), cudaMemcpyDeviceToHost, st), "D2H");
        if (dT) RGF_CUDA(cudaMemcpyAsync(dT, dG.p, ng * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H");
    }
    RGF_CUDA(cudaStreamSynchronize(st), "rgf_conductance");
    std::memcpy(T, hT.data(), nchains * sizeof(double));
    if (chain_status) std::memcpy(chain_status, hs.data(), nchains * sizeof(int32_t));
    for (int i = 0; i < nchains; ++i)
        if (hs[i] != RGF_OK)
            return fail((rgf_status)hs[i], std::string("chain ") + std::to_string(i) + ": " +
                                               rgf_status_str(hs[i]));
    return RGF_OK;
}

struct StreamGuard {
    cudaStream_t st = nullptr;
    ~StreamGuard() {
        if (st) cudaStreamDestroy(st);
    }
};

}  // namespace

namespace rgf {
// Lets other translation units of the library report through rgf_last_error.
void set_last_error(const std::string& msg) { g_last_error = msg; }
}  // namespace rgf

extern "C" {

const char* rgf_version(void) { return "rgf-gb300 0.1"; }

rgf_status rgf_profile_enable(int on) {
    g_prof.on = on != 0;
    g_prof.recorded = false;
    return RGF_OK;
}

rgf_status rgf_profile_read_phases(double* ms) {
    if (!ms) return fail(RGF_EINVAL, "ms is NULL");
    if (!g_prof.on || !g_prof.recorded) return fail(RGF_EINVAL, "no profiled call recorded");
    RGF_CUDA(cudaEventSynchronize(g_prof.ev[kProfEvents - 1]), "cudaEventSynchronize");
    for (int i = 0; i + 1 < kProfEvents; ++i) {
        float a = 0.f;
        RGF_CUDA(cudaEventElapsedTime(&a, g_prof.ev[i], g_prof.ev[i + 1]), "cudaEventElapsedTime");
        ms[i] = a;
    }
    return RGF_OK;
}

rgf_status rgf_profile_read(double* ms_lead, double* ms_sweep) {
    double ms[kProfEvents - 1];
    rgf_status s = rgf_profile_read_phases(ms);
    if (s != RGF_OK) return s;
    if (ms_lead) *ms_lead = ms[0];
    if (ms_sweep) *ms_sweep = ms[1] + ms[2] + ms[3];
    return RGF_OK;
}

rgf_status rgf_set_lead_controls(int max_iter, double residual_tol) {
    if (max_iter < 1 || max_iter > 100000 || !(residual_tol >= 0.0))
        return fail(RGF_EINVAL, "max_iter must be in [1, 100000] and residual_tol >= 0");
    rgf::set_lead_controls(rgf::LeadControls{max_iter, residual_tol});
    return RGF_OK;
}

const char* rgf_last_error(void) { return g_last_error.c_str(); }

const char* rgf_status_str(int s) {
    switch (s) {
        case RGF_OK: return "RGF_OK";
        case RGF_EINVAL: return "RGF_EINVAL: invalid argument";
        case RGF_ENOMEM: return "RGF_ENOMEM: out of memory";
        case RGF_ECUDA: return "RGF_ECUDA: CUDA runtime error";
        case RGF_ENOCONV: return "RGF_ENOCONV: lead decimation did not converge";
        case RGF_ESINGULAR: return "RGF_ESINGULAR: zero pivot in a slice inverse";
        case RGF_ENONFINITE: return "RGF_ENONFINITE: non-finite value";
        case RGF_ETIMEOUT: return "RGF_ETIMEOUT: device wait timed out";
        case RGF_EBOUNDS: return "RGF_EBOUNDS: T outside [0, n_ch]; accuracy lost at this precision";
        default: return "unknown rgf_status";
    }
}

rgf_status rgf_generate_onsite(const rgf_ribbon_desc* d, double* onsite_out, uint8_t* removed_out) {
    rgf_status s = check_desc(d);
    if (s != RGF_OK) return s;
    const int N = d->N, M = 2 * N;
    const size_t n = (size_t)d->L * M;
    if (onsite_out) {
        if (d->onsite) {
            std::memcpy(onsite_out, d->onsite, n * sizeof(double));
        } else {
            for (size_t i = 0; i < n; ++i)
                onsite_out[i] = d->anderson_W * (2.0 * uniform01(d->seed, i) - 1.0);
        }
    }
    if (removed_out) {
        if (d->removed) {
            std::memcpy(removed_out, d->removed, n);
        } else {
            std::memset(removed_out, 0, n);
            if (d->edge_p > 0.0) {
                const int rows[2] = {0, N - 1};
                for (int cell = 0; cell < d->L; ++cell)
                    for (int r = 0; r < 2; ++r) {
                        if (r == 1 && rows[1] == rows[0]) break;
                        for (int k = 0; k < 2; ++k) {
                            size_t i = (size_t)cell * M + 2 * rows[r] + k;
                            removed_out[i] = uniform01(d->edge_seed, i) < d->edge_p ? 1 : 0;
                        }
                    }
            }
        }
    }
    return RGF_OK;
}

rgf_status rgf_build_ribbon(const rgf_ribbon_desc* d, rgf_ribbon** out) {
    if (!out) return fail(RGF_EINVAL, "out is NULL");
    rgf_status s = check_desc(d);
    if (s != RGF_OK) return s;
    const size_t n = (size_t)d->L * 2 * d->N;
    std::vector<double> eps(n);
    std::vector<uint8_t> rem(n);
    rgf_generate_onsite(d, eps.data(), rem.data());
    bool any_rem = false;
    for (size_t i = 0; i < n; ++i) any_rem |= rem[i] != 0;
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(eps[i])) return fail(RGF_EINVAL, "non-finite on-site energy");
    rgf_ribbon* r = new (std::nothrow) rgf_ribbon();
    if (!r) return fail(RGF_ENOMEM, "host allocation failed");
    r->N = d->N;
    r->L = d->L;
    r->t = d->t;
    r->eps = nullptr;
    r->rem = nullptr;
    cudaGetDevice(&r->device);
    cudaError_t e = cudaMalloc(&r->eps, n * sizeof(double));
    if (e == cudaSuccess && any_rem) e = cudaMalloc(&r->rem, n);
    if (e == cudaSuccess) e = cudaMemcpy(r->eps, eps.data(), n * sizeof(double), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && any_rem) e = cudaMemcpy(r->rem, rem.data(), n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        rgf_free_ribbon(r);
        return e == cudaErrorMemoryAllocation ? fail(RGF_ENOMEM, "cudaMalloc(ribbon) failed")
                                              : cuda_fail(e, "ribbon upload");
    }
    *out = r;
    return RGF_OK;
}

rgf_status rgf_build_ribbon_dev(int N, int L, double t, const double* onsite_dev,
                                const uint8_t* removed_dev, void* stream, rgf_ribbon** out) {
    if (!out || !onsite_dev) return fail(RGF_EINVAL, "NULL argument");
    if (N < 2 || N > 2047 || L < 1 || !std::isfinite(t) || t == 0.0)
        return fail(RGF_EINVAL, "bad N, L or t");
    const size_t n = (size_t)L * 2 * N;
    cudaStream_t st = (cudaStream_t)stream;
    rgf_ribbon* r = new (std::nothrow) rgf_ribbon();
    if (!r) return fail(RGF_ENOMEM, "host allocation failed");
    r->N = N;
    r->L = L;
    r->t = t;
    r->eps = nullptr;
    r->rem = nullptr;
    cudaGetDevice(&r->device);
    cudaError_t e = cudaMalloc(&r->eps, n * sizeof(double));
    if (e == cudaSuccess && removed_dev) e = cudaMalloc(&r->rem, n);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(r->eps, onsite_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && removed_dev)
        e = cudaMemcpyAsync(r->rem, removed_dev, n, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        rgf_free_ribbon(r);
        return cuda_fail(e, "rgf_build_ribbon_dev");
    }
    *out = r;
    return RGF_OK;
}

void rgf_free_ribbon(rgf_ribbon* r) {
    if (!r) return;
    if (r->eps) cudaFree(r->eps);
    if (r->rem) cudaFree(r->rem);
    delete r;
}

rgf_status rgf_lead_selfenergy(int N, double t, const double* E, int nE, double eta, int side,
                               double* sigma, int* iters) {
    if (N < 2 || N > 2047 || nE < 0 || !E || !sigma || (side != 0 && side != 1) ||
        !(eta > 0.0) || !std::isfinite(t) || t == 0.0)
        return fail(RGF_EINVAL, "bad argument to rgf_lead_selfenergy");
    if (nE == 0) return RGF_OK;
    for (int i = 0; i < nE; ++i)
        if (!std::isfinite(E[i])) return fail(RGF_EINVAL, "non-finite energy");
    const int KL = rgf::col_KL(N), KR = rgf::col_KR(N), M = 2 * N;
    std::vector<rgf::LeadDev> leads(nE);
    size_t ws = 0, outn = 0;
    for (int i = 0; i < nE; ++i) {
        leads[i].N = N;
        leads[i].t = t;
        leads[i].E = E[i];
        leads[i].off = outn;
        leads[i].ws_off = ws;
        outn += rgf::lead_out_elems(N);
        ws += rgf::lead_ws_elems(N);
    }
    cudaStream_t st = 0;
    DevBuf dleads, dws, dout, dst, dit;
    RGF_CUDA(dleads.alloc(nE * sizeof(rgf::LeadDev), st), "cudaMallocAsync");
    RGF_CUDA(dws.alloc(ws * 16, st), "cudaMallocAsync");
    RGF_CUDA(dout.alloc(outn * 16, st), "cudaMallocAsync");
    RGF_CUDA(dst.alloc(2 * nE * sizeof(int), st), "cudaMallocAsync");
    RGF_CUDA(dit.alloc(2 * nE * sizeof(int), st), "cudaMallocAsync");
    RGF_CUDA(cudaMemcpyAsync(dleads.p, leads.data(), nE * sizeof(rgf::LeadDev),
                             cudaMemcpyHostToDevice, st), "cudaMemcpyAsync");
    RGF_CUDA(rgf::launch_lead((rgf::LeadDev*)dleads.p, nE, KL, eta, dws.p, dout.p, (int*)dst.p,
                              (int*)dit.p, st), "lead decimation launch");
    std::vector<double> hout(outn * 2);
    std::vector<int> hst(2 * nE), hit(2 * nE);
    RGF_CUDA(cudaMemcpyAsync(hout.data(), dout.p, outn * 16, cudaMemcpyDeviceToHost, st), "D2H");
    RGF_CUDA(cudaMemcpyAsync(hst.data(), dst.p, 2 * nE * sizeof(int), cudaMemcpyDeviceToHost, st), "D2H");
    RGF_CUDA(cudaMemcpyAsync(hit.data(), dit.p, 2 * nE * sizeof(int), cudaMemcpyDeviceToHost, st), "D2H");
    RGF_CUDA(cudaStreamSynchronize(st), "lead decimation");
    rgf_status result = RGF_OK;
    const size_t MM = (size_t)M * M;
    for (int i = 0; i < nE; ++i) {
        double* S = sigma + 2 * MM * i;
        int ok = hst[2 * i + side] == 0;
        if (iters) iters[i] = hit[2 * i + side];
        if (!ok) {
            result = fail(RGF_ENOCONV, "lead decimation did not converge at E = " +
                                           std::to_string(E[i]));
            for (size_t e = 0; e < 2 * MM; ++e) S[e] = NAN;
            continue;
        }
        std::memset(S, 0, 2 * MM * sizeof(double));
        const double* blk = hout.data() + 2 * leads[i].off + (side ? 2 * (size_t)KL * KL : 0);
        const int K = side ? KR : KL, c = side ? 3 : 0;
        for (int a = 0; a < K; ++a)
            for (int b = 0; b < K; ++b) {
                size_t oa = 4 * a + c, ob = 4 * b + c;
                S[2 * (oa * M + ob)] = blk[2 * ((size_t)a * K + b)];
                S[2 * (oa * M + ob) + 1] = blk[2 * ((size_t)a * K + b) + 1];
            }
    }
    return result;
}

rgf_status rgf_conductance_dev(const rgf_ribbon* const* rib, const double* E_dev, int nchains,
                               double eta_device, double eta_lead, int precision, void* stream,
                               double* T_dev, int32_t* status_dev) {
    return run_path(rib, E_dev, nchains, eta_device, eta_lead, precision, (cudaStream_t)stream,
                    T_dev, status_dev);
}

rgf_status rgf_conductance(const rgf_ribbon* const* rib, const double* E, int nchains,
                           double eta_device, double eta_lead, int precision, double* T,
                           int32_t* chain_status) {
    return run_host(rib, E, nchains, eta_device, eta_lead, precision, T, chain_status);
}

rgf_status rgf_conductance_grad_dev(const rgf_ribbon* const* rib, const double* E_dev,
                                    int nchains, double eta_device, double eta_lead,
                                    int precision, int ckpt_stride, const double* weights_dev,
                                    void* stream, double* T_dev, double* dT_dev,
                                    int32_t* status_dev) {
    if (nchains < 0) return fail(RGF_EINVAL, "nchains < 0");
    if (nchains == 0) return RGF_OK;
    if (!rib || !dT_dev) return fail(RGF_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (!weights_dev)
        return run_path(rib, E_dev, nchains, eta_device, eta_lead, precision, st, T_dev,
                        status_dev, dT_dev, ckpt_stride);
    for (int c = 0; c < nchains; ++c) {
        if (!rib[c]) return fail(RGF_EINVAL, "NULL ribbon");
        if (rib[c]->N != rib[0]->N || rib[c]->L != rib[0]->L)
            return fail(RGF_EINVAL, "weights_dev needs ribbons of one size (N, L)");
    }
    const size_t n = (size_t)rib[0]->L * 2 * rib[0]->N;
    DevBuf per;
    RGF_CUDA(per.alloc((size_t)nchains * n * sizeof(double), st), "cudaMallocAsync(gradients)");
    rgf_status s = run_path(rib, E_dev, nchains, eta_device, eta_lead, precision, st, T_dev,
                            status_dev, (double*)per.p, ckpt_stride);
    if (s != RGF_OK) return s;
    weighted_chain_sum<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const double*)per.p, weights_dev,
                                                                    nchains, n, dT_dev);
    RGF_CUDA(cudaGetLastError(), "weighted_chain_sum launch");
    return RGF_OK;
}

rgf_status rgf_ldos(const rgf_ribbon* const* rib, const double* E, int nchains, double eta_device,
                    double eta_lead, int precision, int ckpt_stride, double* T, double* rho,
                    int32_t* chain_status) {
    if (nchains > 0 && !rho) return fail(RGF_EINVAL, "rho is NULL");
    return run_host(rib, E, nchains, eta_device, eta_lead, precision, T, chain_status, rho,
                    ckpt_stride, rgf::OUT_LDOS);
}

rgf_status rgf_conductance_grad(const rgf_ribbon* const* rib, const double* E, int nchains,
                                double eta_device, double eta_lead, int precision,
                                int ckpt_stride, double* T, double* dT_deps,
                                int32_t* chain_status) {
    if (nchains > 0 && !dT_deps) return fail(RGF_EINVAL, "dT_deps is NULL");
    return run_host(rib, E, nchains, eta_device, eta_lead, precision, T, chain_status, dT_deps,
                    ckpt_stride);
}

}  // extern "C"
