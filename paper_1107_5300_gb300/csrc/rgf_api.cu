// rgf_api.cu -- host side of the C ABI declared in include/rgf.h: ribbon
// instances, argument checks, workspace, launch order, status reporting.
//
// Call flow of rgf_conductance (the paper's step list: input and defects ->
// lead self-energies -> recursion on the device -> conductance):
//   1. one lead problem per chain (pristine ribbon of the chain's width at the
//      chain's energy), decimated on the device (rgf_lead.cu);
//   2. the column-sliced recursion as two halves per chain, one from each
//      lead, joined by one Dyson step, and the trace (rgf_half.cuh: end-column
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

// external: record as an event node of a graph being captured on `st`.
cudaError_t prof_record(int i, cudaStream_t st, bool external = false) {
    if (!g_prof.on) return cudaSuccess;
    if (!g_prof.ev[i]) {
        cudaError_t e = cudaEventCreate(&g_prof.ev[i]);
        if (e != cudaSuccess) return e;
    }
    return external ? cudaEventRecordWithFlags(g_prof.ev[i], st, cudaEventRecordExternal)
                    : cudaEventRecord(g_prof.ev[i], st);
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

bool valid_precision(int p) {
    return p == RGF_FP64 || p == RGF_MIXED || p == RGF_MIXED_TC || p == RGF_FP64_TC;
}
bool tc_precision(int p) { return p == RGF_MIXED_TC || p == RGF_FP64_TC; }
// The precision a tensor-core precision's chains run in on the pipes.
int pipes_precision(int p) { return p == RGF_FP64_TC ? RGF_FP64 : p == RGF_MIXED_TC ? RGF_MIXED : p; }

// Schedule of the forward sweep and the tuning tables (process-wide).  A
// table, per precision, maps the column size K = ceil(N/2) of a chain to its
// schedule: the first entry with K <= K_max, else the last entry; an empty
// table means the default (tensor cores with the _TC precisions, widest panel,
// pair steps).  The autotuner's timing runs force one entry for every chain
// (thread-local).
std::mutex g_tune_mu;
std::vector<rgf_tune_entry> g_tune[4];
int g_schedule = RGF_SCHED_PHASED;
thread_local const rgf_tune_entry* g_force = nullptr;
thread_local int g_force_schedule = -1;
int g_domains = 2;                       // domains per chain; 0 = automatic
thread_local int g_force_domains = 0;

// Domains per chain for a call (forward sweep): forced (>= 2), else as many as
// leave every chain one SM per domain, but at most ncol / 32: the joins run as
// a tree, log2 of the interior domains deep, each level a few tens of column
// steps' worth, so domains of 32 columns or more keep them a minor part.  At
// most ncol / 2 (every domain two columns or more).
int domains_for(int requested, int nchains, int ncol_min, int nsm) {
    int d;
    if (requested >= 2) {
        d = requested;
    } else {
        const int per = nchains > 0 ? nsm / nchains : 2;
        d = std::max(2, std::min(per, ncol_min / 32));
    }
    return std::max(2, std::min(d, ncol_min / 2));
}

rgf_tune_entry default_entry() { return rgf_tune_entry{0x7fffffff, RGF_ENGINE_TENSOR, 0, 1}; }

rgf_tune_entry lookup_tune(int precision, int K) {
    if (g_force) return *g_force;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const std::vector<rgf_tune_entry>& t = g_tune[precision];
    if (t.empty()) return default_entry();
    for (const rgf_tune_entry& e : t)
        if (K <= e.K_max) return e;
    return t.back();
}

// One launch group of the forward sweep: the chains that run on one engine,
// longest first.  Chains of a tensor-core precision tuned to the pipes form a
// second group that runs as the matching pipes precision (RGF_MIXED_TC as
// RGF_MIXED, RGF_FP64_TC as RGF_FP64: same arithmetic, products on the pipes).
struct Group {
    int precision = 0;
    int Kmax = 1;
    std::vector<int> order;
};

struct Plan {
    std::vector<rgf::ChainDev> chains;
    std::vector<rgf::LeadDev> leads;
    std::vector<int> order;          // all chains, longest first (gradient sweep)
    std::vector<Group> groups;       // forward sweep
    int ndom = 2;                    // domains per chain (forward sweep)
    std::vector<int> seg_cols;
    size_t ws_elems = 0, lead_ws_elems = 0, lead_out_elems = 0, grad_elems = 0;
    int Kmax = 1;
};

// grad: size the gradient workspace with checkpoints every ckpt_stride cells
// (<= 0: ceil(sqrt(L))).  precision: that of the call (picks the tuning table
// and the forward sweep's groups).
rgf_status make_plan(const rgf_ribbon* const* rib, int nchains, int precision, Plan& pl,
                     bool grad = false, int ckpt_stride = 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    pl.chains.resize(nchains);
    pl.leads.resize(nchains);
    pl.seg_cols.resize(nchains);
    std::vector<double> cost(nchains);
    std::vector<int> engine(nchains, 0);
    if (!grad) {
        int ncol_min = 1 << 30, nsm = 1;
        for (int c = 0; c < nchains; ++c) {
            if (!rib[c]) return fail(RGF_EINVAL, "rib[" + std::to_string(c) + "] is NULL");
            ncol_min = std::min(ncol_min, 4 * rib[c]->L);
        }
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) nsm = 1;
        int req = g_force_domains;
        if (!req) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            req = g_domains;
        }
        pl.ndom = domains_for(req, nchains, ncol_min, nsm);
    }
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
        rgf::default_sched(ch);
        if (grad) {
            int stride = ckpt_stride > 0 ? std::min(ckpt_stride, r->L)
                                         : std::max(1, (int)std::ceil(std::sqrt((double)r->L)));
            pl.seg_cols[c] = 4 * stride;
            pl.ws_elems += rgf::grad_ws_elems(r->N, r->L, pl.seg_cols[c]);
            pl.grad_elems += (size_t)r->L * 2 * r->N;
        } else {
            const rgf_tune_entry te = lookup_tune(precision, rgf::col_KL(r->N));
            ch.panel = (int8_t)te.panel;
            ch.pairs = (int8_t)(te.pairs != 0);
            ch.tc = (int8_t)(tc_precision(precision) && te.engine == RGF_ENGINE_TENSOR &&
                             rgf::tc_layout_fits(rgf::col_KL(r->N)));
            engine[c] = ch.tc;
            pl.seg_cols[c] = 0;
            pl.ws_elems += rgf::chain_ws_elems(r->N, pl.ndom);
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
    // longest processing time first: the queue (or the block scheduler) then
    // hands the remaining work to whichever SM frees up first
    pl.order.resize(nchains);
    for (int c = 0; c < nchains; ++c) pl.order[c] = c;
    std::stable_sort(pl.order.begin(), pl.order.end(),
                     [&](int a, int b) { return cost[a] > cost[b]; });
    if (!grad) {
        const bool split = tc_precision(precision);
        for (int pass = 0; pass < (split ? 2 : 1); ++pass) {
            Group g;
            g.precision = split ? (pass == 0 ? precision : pipes_precision(precision)) : precision;
            for (int c : pl.order)
                if (!split || engine[c] == (pass == 0 ? 1 : 0)) {
                    g.order.push_back(c);
                    g.Kmax = std::max(g.Kmax, rgf::col_KL(pl.chains[c].N));
                }
            if (!g.order.empty()) pl.groups.push_back(std::move(g));
        }
    }
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

// The device side of a plan: one allocation holding the descriptors, the
// groups' orders and work queues, the lead buffers and the sweep workspace
// (each part 256-byte aligned).
struct DevLayout {
    size_t o_chain = 0, o_lead = 0, o_order = 0, o_seg = 0, o_queue = 0, o_lst = 0, o_lws = 0,
           o_lout = 0, o_ws = 0, total = 0, queue_bytes = 0, hdr_bytes = 0;
};
inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

DevLayout layout_of(const Plan& pl) {
    const size_t n = pl.chains.size();
    DevLayout d;
    d.o_chain = 0;
    d.o_lead = up256(n * sizeof(rgf::ChainDev));
    d.o_order = d.o_lead + up256(n * sizeof(rgf::LeadDev));
    d.o_seg = d.o_order + up256(n * sizeof(int));   // groups' orders, concatenated
    d.hdr_bytes = d.o_seg + n * sizeof(int);
    d.o_queue = up256(d.hdr_bytes);
    d.queue_bytes = std::max<size_t>(1, pl.groups.size()) * rgf::batch_queue_ints((int)n) * sizeof(int);
    d.o_lst = d.o_queue + up256(d.queue_bytes);
    d.o_lws = d.o_lst + up256(2 * n * sizeof(int));
    d.o_lout = d.o_lws + up256(pl.lead_ws_elems * 16);
    d.o_ws = d.o_lout + up256(pl.lead_out_elems * 16);
    d.total = d.o_ws + std::max<size_t>(pl.ws_elems, 1) * 16;
    return d;
}

// Host image of the header part of the layout (descriptors, orders, segments).
std::vector<unsigned char> header_of(const Plan& pl, const DevLayout& d) {
    std::vector<unsigned char> h(d.hdr_bytes, 0);
    const size_t n = pl.chains.size();
    std::memcpy(h.data() + d.o_chain, pl.chains.data(), n * sizeof(rgf::ChainDev));
    std::memcpy(h.data() + d.o_lead, pl.leads.data(), n * sizeof(rgf::LeadDev));
    if (pl.groups.empty()) {
        std::memcpy(h.data() + d.o_order, pl.order.data(), n * sizeof(int));
    } else {
        size_t k = 0;
        for (const Group& g : pl.groups) {
            std::memcpy(h.data() + d.o_order + k * sizeof(int), g.order.data(), g.order.size() * sizeof(int));
            k += g.order.size();
        }
    }
    std::memcpy(h.data() + d.o_seg, pl.seg_cols.data(), n * sizeof(int));
    return h;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    return n;
}

// Sets the shared-memory limits of every kernel a plan's forward sweep
// launches (before a stream capture, and by every launcher anyway).
cudaError_t configure_groups(const Plan& pl) {
    for (const Group& g : pl.groups) {
        cudaError_t e = rgf::configure_sweep(g.precision, g.Kmax);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Enqueues the forward path of a plan on `st`: energies into the descriptors,
// lead decimation, then per group the persistent batch kernel (or, with the
// phased schedule, the three launches; all groups' preparations, then their
// recursions, then their joins).  base: the plan's device allocation.
// prof: 0 no profile events, 1 events on the stream, 2 event nodes of the
// graph being captured on `st`.
rgf_status enqueue_forward(const Plan& pl, const DevLayout& d, unsigned char* base,
                           const double* E_dev, double eta_device, double eta_lead,
                           cudaStream_t st, double* T_dev, int32_t* status_dev, int schedule,
                           int prof) {
    const int n = (int)pl.chains.size();
    auto* dchains = (rgf::ChainDev*)(base + d.o_chain);
    auto* dleads = (rgf::LeadDev*)(base + d.o_lead);
    auto* dorder = (int*)(base + d.o_order);
    auto* dqueue = (int*)(base + d.o_queue);
    auto* dlst = (int*)(base + d.o_lst);
    void* dlws = base + d.o_lws;
    void* dlout = base + d.o_lout;
    void* dws = base + d.o_ws;
    auto rec = [&](int i) { return prof ? prof_record(i, st, prof == 2) : cudaSuccess; };
    fill_energy<<<(n + 255) / 256, 256, 0, st>>>(dchains, dleads, E_dev, n);
    RGF_CUDA(cudaGetLastError(), "fill_energy launch");
    RGF_CUDA(rec(0), "cudaEventRecord");
    RGF_CUDA(rgf::launch_lead(dleads, n, pl.Kmax, eta_lead, dlws, dlout, dlst, nullptr, st),
             "lead decimation launch");
    RGF_CUDA(rec(1), "cudaEventRecord");
    if (schedule == RGF_SCHED_PERSISTENT && pl.ndom == 2) {
        RGF_CUDA(cudaMemsetAsync(dqueue, 0, d.queue_bytes, st), "cudaMemsetAsync(work queue)");
        RGF_CUDA(rec(2), "cudaEventRecord");
        const int nsm = sm_count();
        size_t k = 0;
        for (size_t gi = 0; gi < pl.groups.size(); ++gi) {
            const Group& g = pl.groups[gi];
            RGF_CUDA(rgf::launch_batch(g.precision, dchains, dorder + k, (int)g.order.size(), g.Kmax,
                                       eta_device, dlout, dlst, dleads, dws, T_dev, status_dev,
                                       dqueue + gi * rgf::batch_queue_ints(n), nsm, st),
                     "persistent sweep launch");
            k += g.order.size();
        }
        RGF_CUDA(rec(3), "cudaEventRecord");
    } else {
        size_t k = 0;
        for (const Group& g : pl.groups) {
            RGF_CUDA(rgf::launch_prep(g.precision, dchains, dorder + k, (int)g.order.size(), g.Kmax,
                                      eta_device, dlout, dlst, dleads, dws, st, pl.ndom),
                     "end-column preparation launch");
            k += g.order.size();
        }
        RGF_CUDA(rec(2), "cudaEventRecord");
        k = 0;
        for (const Group& g : pl.groups) {
            RGF_CUDA(rgf::launch_half(g.precision, dchains, dorder + k, (int)g.order.size(), g.Kmax,
                                      eta_device, dlout, dlst, dleads, dws, st, pl.ndom),
                     "half sweep launch");
            k += g.order.size();
        }
        RGF_CUDA(rec(3), "cudaEventRecord");
        k = 0;
        for (const Group& g : pl.groups) {
            RGF_CUDA(rgf::launch_merge(g.precision, dchains, dorder + k, (int)g.order.size(), g.Kmax,
                                       eta_device, dlout, dlst, dleads, dws, T_dev, status_dev, st,
                                       pl.ndom),
                     "merge launch");
            k += g.order.size();
        }
    }
    RGF_CUDA(rec(4), "cudaEventRecord");
    if (prof == 1 && g_prof.on) g_prof.recorded = true;
    return RGF_OK;
}

rgf_status check_call(const rgf_ribbon* const* rib, const void* E_dev, const void* T_dev,
                      int nchains, int precision, double eta_device, double eta_lead) {
    if (nchains < 0) return fail(RGF_EINVAL, "nchains < 0");
    if (nchains > 0 && (!rib || !E_dev || !T_dev)) return fail(RGF_EINVAL, "NULL argument");
    if (!valid_precision(precision))
        return fail(RGF_EINVAL, "unknown precision");
    if (!(eta_device >= 0.0) || !(eta_lead > 0.0) || !std::isfinite(eta_device) ||
        !std::isfinite(eta_lead))
        return fail(RGF_EINVAL, "eta_device must be >= 0 and eta_lead > 0 (finite)");
    return RGF_OK;
}

// Runs the whole path on `st`: lead decimation, then the forward sweep (or,
// with dT_dev, the checkpointed two-sided gradient sweep).  E_dev, T_dev, status_dev,
// dT_dev: device.
rgf_status run_path(const rgf_ribbon* const* rib, const double* E_dev, int nchains,
                    double eta_device, double eta_lead, int precision, cudaStream_t st,
                    double* T_dev, int32_t* status_dev, double* dT_dev = nullptr,
                    int ckpt_stride = 0, int out_mode = rgf::OUT_GRAD) {
    rgf_status s = check_call(rib, E_dev, T_dev, nchains, precision, eta_device, eta_lead);
    if (s != RGF_OK || nchains == 0) return s;
    const bool grad = dT_dev != nullptr;
    Plan pl;
    s = make_plan(rib, nchains, precision, pl, grad, ckpt_stride);
    if (s != RGF_OK) return s;
    const DevLayout d = layout_of(pl);
    const std::vector<unsigned char> hdr = header_of(pl, d);
    DevBuf dmem;
    cudaError_t ae = dmem.alloc(d.total, st);
    if (ae == cudaErrorMemoryAllocation) return fail(RGF_ENOMEM, "workspace allocation failed");
    RGF_CUDA(ae, "cudaMallocAsync(workspace)");
    unsigned char* base = (unsigned char*)dmem.p;
    RGF_CUDA(cudaMemcpyAsync(base, hdr.data(), hdr.size(), cudaMemcpyHostToDevice, st),
             "cudaMemcpyAsync(descriptors)");
    if (!grad) {
        int sched = g_force_schedule;
        if (sched < 0) {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            sched = g_schedule;
        }
        return enqueue_forward(pl, d, base, E_dev, eta_device, eta_lead, st, T_dev, status_dev,
                               sched, 1);
    }
    RGF_CUDA(cudaMemsetAsync(dT_dev, 0, pl.grad_elems * sizeof(double), st), "cudaMemsetAsync");
    double* dgrad = (out_mode & rgf::OUT_GRAD) ? dT_dev : nullptr;
    double* drho = (out_mode & rgf::OUT_LDOS) ? dT_dev : nullptr;
    auto* dchains = (rgf::ChainDev*)(base + d.o_chain);
    auto* dleads = (rgf::LeadDev*)(base + d.o_lead);
    auto* dorder = (int*)(base + d.o_order);
    auto* dseg = (int*)(base + d.o_seg);
    auto* dlst = (int*)(base + d.o_lst);
    fill_energy<<<(nchains + 255) / 256, 256, 0, st>>>(dchains, dleads, E_dev, nchains);
    RGF_CUDA(cudaGetLastError(), "fill_energy launch");
    RGF_CUDA(prof_record(0, st), "cudaEventRecord");
    RGF_CUDA(rgf::launch_lead(dleads, nchains, pl.Kmax, eta_lead, base + d.o_lws, base + d.o_lout,
                              dlst, nullptr, st),
             "lead decimation launch");
    RGF_CUDA(prof_record(1, st), "cudaEventRecord");
    RGF_CUDA(prof_record(2, st), "cudaEventRecord");
    RGF_CUDA(rgf::launch_grad(precision, dchains, dorder, nchains, pl.Kmax, eta_device,
                              base + d.o_lout, dlst, dleads, base + d.o_ws, dseg, T_dev, dgrad,
                              drho, out_mode, status_dev, st),
             "gradient sweep launch");
    RGF_CUDA(prof_record(3, st), "cudaEventRecord");
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

rgf_status rgf_set_schedule(int schedule) {
    if (schedule != RGF_SCHED_PERSISTENT && schedule != RGF_SCHED_PHASED)
        return fail(RGF_EINVAL, "unknown schedule");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_schedule = schedule;
    return RGF_OK;
}

rgf_status rgf_set_domains(int ndom) {
    if (ndom != 0 && (ndom < 2 || ndom > 4096)) return fail(RGF_EINVAL, "ndom must be 0 or in [2, 4096]");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_domains = ndom;
    return RGF_OK;
}

int rgf_get_domains(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_domains;
}

int rgf_auto_domains(int nchains, int ncol_min, int nsm) {
    return domains_for(0, nchains, std::max(ncol_min, 4), std::max(nsm, 1));
}

int rgf_get_schedule(void) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    return g_schedule;
}

rgf_status rgf_set_tuning(int precision, const rgf_tune_entry* table, int n) {
    if (!valid_precision(precision))
        return fail(RGF_EINVAL, "unknown precision");
    if (n < 0 || n > RGF_TUNE_MAX_ENTRIES || (n > 0 && !table))
        return fail(RGF_EINVAL, "n must be in [0, RGF_TUNE_MAX_ENTRIES] with a table");
    for (int i = 0; i < n; ++i) {
        const rgf_tune_entry& e = table[i];
        if (e.K_max < 1 || (i > 0 && e.K_max <= table[i - 1].K_max))
            return fail(RGF_EINVAL, "K_max must be >= 1 and strictly increasing");
        if (e.engine != RGF_ENGINE_PIPES && e.engine != RGF_ENGINE_TENSOR)
            return fail(RGF_EINVAL, "engine must be RGF_ENGINE_PIPES or RGF_ENGINE_TENSOR");
        if (e.panel != 0 && e.panel != 2 && e.panel != 4 && e.panel != 8 && e.panel != 16)
            return fail(RGF_EINVAL, "panel must be 0, 2, 4, 8 or 16");
        if (e.pairs != 0 && e.pairs != 1) return fail(RGF_EINVAL, "pairs must be 0 or 1");
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[precision].assign(table, table + n);
    return RGF_OK;
}

rgf_status rgf_get_tuning(int precision, rgf_tune_entry* table, int cap, int* n) {
    if (!valid_precision(precision))
        return fail(RGF_EINVAL, "unknown precision");
    if (!n || cap < 0 || (cap > 0 && !table)) return fail(RGF_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const std::vector<rgf_tune_entry>& t = g_tune[precision];
    *n = (int)t.size();
    if ((int)t.size() > cap) return fail(RGF_EINVAL, "table capacity too small");
    std::copy(t.begin(), t.end(), table);
    return RGF_OK;
}

rgf_status rgf_tune_lookup(int precision, int N, rgf_tune_entry* out) {
    if (!valid_precision(precision))
        return fail(RGF_EINVAL, "unknown precision");
    if (!out || N < 2) return fail(RGF_EINVAL, "bad argument");
    *out = lookup_tune(precision, rgf::col_KL(N));
    return RGF_OK;
}

rgf_status rgf_autotune(int precision, const int* N, int nN, int cells, int reps,
                        rgf_tune_entry* best, double* ms, int* ncand) {
    if (!valid_precision(precision))
        return fail(RGF_EINVAL, "unknown precision");
    if (nN < 1 || nN > RGF_TUNE_MAX_ENTRIES || !N || !best || cells < 1 || reps < 1)
        return fail(RGF_EINVAL, "bad argument to rgf_autotune");
    for (int i = 0; i < nN; ++i)
        if (N[i] < 2 || N[i] > 2047) return fail(RGF_EINVAL, "N must be in [2, 2047]");
    // widths by column size; idx[b] = the caller's index of the b-th
    std::vector<int> idx(nN);
    for (int i = 0; i < nN; ++i) idx[i] = i;
    std::sort(idx.begin(), idx.end(), [&](int a, int b) { return rgf::col_KL(N[a]) < rgf::col_KL(N[b]); });
    std::vector<int> Ns(nN);
    for (int b = 0; b < nN; ++b) Ns[b] = N[idx[b]];
    for (int i = 1; i < nN; ++i)
        if (rgf::col_KL(Ns[i]) == rgf::col_KL(Ns[i - 1]))
            return fail(RGF_EINVAL, "two widths with the same column size ceil(N/2)");
    // the candidates: engine x panel width x pair steps
    std::vector<rgf_tune_entry> cand;
    const int engines = tc_precision(precision) ? 2 : 1;
    for (int en = 0; en < engines; ++en)
        for (int panel : {16, 8, 4})
            for (int pairs : {1, 0})
                cand.push_back(rgf_tune_entry{0, tc_precision(precision) ? 1 - en : 0, panel, pairs});
    if (ncand) *ncand = (int)cand.size();
    const bool prof_was = g_prof.on;
    g_prof.on = true;
    rgf_status result = RGF_OK;
    std::vector<rgf_tune_entry> table;
    for (int b = 0; b < nN && result == RGF_OK; ++b) {
        // one chain: an Anderson-disordered ribbon of `cells` unit cells at
        // 0.3 eV; the time of its half sweeps (the three-launch schedule's
        // middle launch, the only step the candidates change)
        rgf_ribbon_desc desc{};
        desc.N = Ns[b];
        desc.L = cells;
        desc.t = -2.7;
        desc.anderson_W = 0.1;
        desc.seed = 12345;
        rgf_ribbon* r = nullptr;
        result = rgf_build_ribbon(&desc, &r);
        if (result != RGF_OK) break;
        double* dE = nullptr;
        double* dT = nullptr;
        const double E = 0.3;
        cudaError_t e = cudaMalloc(&dE, sizeof(double));
        if (e == cudaSuccess) e = cudaMalloc(&dT, sizeof(double));
        if (e == cudaSuccess) e = cudaMemcpy(dE, &E, sizeof(double), cudaMemcpyHostToDevice);
        double best_ms = INFINITY;
        rgf_tune_entry win = cand[0];
        for (size_t ci = 0; ci < cand.size() && e == cudaSuccess && result == RGF_OK; ++ci) {
            double t_min = INFINITY;
            for (int rep = 0; rep <= reps && result == RGF_OK; ++rep) {   // rep 0: warm-up
                g_force = &cand[ci];
                g_force_schedule = RGF_SCHED_PHASED;
                g_force_domains = 2;
                result = run_path(&r, dE, 1, 1e-8, 1e-8, precision, 0, dT, nullptr);
                g_force = nullptr;
                g_force_schedule = -1;
                g_force_domains = 0;
                if (result != RGF_OK) break;
                double ph[kProfEvents - 1];
                result = rgf_profile_read_phases(ph);
                if (rep > 0) t_min = std::min(t_min, ph[2]);
            }
            if (ms) ms[(size_t)idx[b] * cand.size() + ci] = t_min;
            if (t_min < best_ms) {
                best_ms = t_min;
                win = cand[ci];
            }
        }
        if (e != cudaSuccess) result = cuda_fail(e, "rgf_autotune buffers");
        if (dE) cudaFree(dE);
        if (dT) cudaFree(dT);
        rgf_free_ribbon(r);
        win.K_max = rgf::col_KL(Ns[b]);
        table.push_back(win);
        best[idx[b]] = win;
    }
    g_prof.on = prof_was;
    g_prof.recorded = false;
    if (result != RGF_OK) return result;
    return rgf_set_tuning(precision, table.data(), (int)table.size());
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Prepared batches: the forward path of a fixed list of chains as one CUDA
// graph.
// ---------------------------------------------------------------------------
struct rgf_batch {
    int device = 0;
    bool profiled = false;   // the graph records the profile events
    Plan plan;
    DevLayout layout;
    unsigned char* mem = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" {

void rgf_batch_free(rgf_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->mem) cudaFree(b->mem);
    delete b;
}

rgf_status rgf_batch_create(const rgf_ribbon* const* rib, const double* E_dev, int nchains,
                            double eta_device, double eta_lead, int precision, double* T_dev,
                            int32_t* status_dev, rgf_batch** out) {
    if (!out) return fail(RGF_EINVAL, "out is NULL");
    *out = nullptr;
    rgf_status s = check_call(rib, E_dev, T_dev, nchains, precision, eta_device, eta_lead);
    if (s != RGF_OK) return s;
    if (nchains == 0) return fail(RGF_EINVAL, "a batch needs at least one chain");
    rgf_batch* b = new (std::nothrow) rgf_batch();
    if (!b) return fail(RGF_ENOMEM, "host allocation failed");
    cudaGetDevice(&b->device);
    s = make_plan(rib, nchains, precision, b->plan);
    if (s != RGF_OK) {
        rgf_batch_free(b);
        return s;
    }
    b->layout = layout_of(b->plan);
    const std::vector<unsigned char> hdr = header_of(b->plan, b->layout);
    cudaError_t e = cudaMalloc(&b->mem, b->layout.total);
    if (e != cudaSuccess) {
        rgf_batch_free(b);
        return e == cudaErrorMemoryAllocation ? fail(RGF_ENOMEM, "batch workspace allocation failed")
                                              : cuda_fail(e, "cudaMalloc(batch)");
    }
    e = cudaMemcpy(b->mem, hdr.data(), hdr.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = configure_groups(b->plan);
    if (e != cudaSuccess) {
        rgf_batch_free(b);
        return cuda_fail(e, "batch set-up");
    }
    // capture the launch sequence on a private stream
    StreamGuard cs;
    e = cudaStreamCreateWithFlags(&cs.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs.st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        rgf_batch_free(b);
        return cuda_fail(e, "stream capture");
    }
    b->profiled = g_prof.on;
    int sched;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        sched = g_schedule;
    }
    s = enqueue_forward(b->plan, b->layout, b->mem, E_dev, eta_device, eta_lead, cs.st, T_dev,
                        status_dev, sched, b->profiled ? 2 : 0);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs.st, &g);
    b->graph = g;
    if (s != RGF_OK) {
        rgf_batch_free(b);
        return s;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
        rgf_batch_free(b);
        return cuda_fail(e, "graph capture");
    }
    *out = b;
    return RGF_OK;
}

rgf_status rgf_batch_launch(rgf_batch* b, void* stream) {
    if (!b || !b->exec) return fail(RGF_EINVAL, "batch is NULL");
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != b->device) return fail(RGF_EINVAL, "batch was created on another device");
    RGF_CUDA(cudaGraphLaunch(b->exec, (cudaStream_t)stream), "cudaGraphLaunch");
    if (b->profiled && g_prof.on) g_prof.recorded = true;
    return RGF_OK;
}

}  // extern "C"
