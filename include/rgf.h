/*
 * rgf.h -- C ABI of the GB300 recursive Green's function (RGF) library.
 *
 * Computes the two-terminal Landauer conductance of armchair graphene
 * nanoribbons (one p orbital per carbon atom, nearest-neighbour hopping t,
 * semi-infinite pristine leads of the same width), following S. Ihnatsenka,
 * Comput. Phys. Commun. 183 (2012) 543:
 *
 *   Eq. 1   G = (E - H)^-1, retarded: E -> E + i*eta
 *   Eq. 2   T = Tr[Gamma_L G_1L Gamma_R G_1L^dagger]   (conductance in 2e^2/h)
 *   Eq. 3   Dyson equation G = G0 + G0 Sigma G, applied slice by slice as
 *   Eqs. 4-5  g_j = (z - H_jj - V^T g_{j-1} V)^-1,   G_1j = G_1,j-1 V g_j
 *
 * with the lead self-energies Sigma_L, Sigma_R included at the first and the
 * last slice (text after Eqs. 4-5), computed here by Lopez Sancho-Rubio
 * decimation, and Gamma = i (Sigma - Sigma^dagger).
 *
 * Geometry and orbital order.  A ribbon has N dimer lines (rows j = 0..N-1)
 * and L unit cells along the transport axis; a unit cell holds M = 2N atoms.
 * Even rows hold atoms at x = 0 and a, odd rows at x = 1.5a and 2.5a (a = C-C
 * distance).  Orbital o = 2*j + k of a cell is the left (k = 0) or right (k = 1)
 * atom of row j.  Per-orbital arrays are row-major [L][2N].
 *
 * Conventions for every entry point:
 *   - Callers own every buffer they pass; the library never keeps a pointer
 *     to caller memory after the call returns (except rgf_build_ribbon_dev,
 *     which documents its own rule).
 *   - Nothing throws or aborts across this ABI.  A call returns RGF_OK or the
 *     first error; rgf_last_error() then gives a message (per thread).
 *   - Calls without a `stream` argument run on the legacy default stream of the
 *     current device and return after the results are on the host.
 *   - "Host" pointers are ordinary CPU memory; "device" pointers are CUDA
 *     global memory of the current device.
 *   - On a failing call, host outputs are left untouched where the error is
 *     caught before launch (RGF_EINVAL, RGF_ENOMEM); per-chain numeric failures
 *     (RGF_ENOCONV, RGF_ESINGULAR, RGF_ENONFINITE, RGF_ETIMEOUT, RGF_EBOUNDS) are reported
 *     per chain in chain_status, that chain's T is NaN, and the other chains'
 *     results are valid.
 */
#ifndef RGF_H
#define RGF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    RGF_OK = 0,
    RGF_EINVAL = 1,      /* bad argument (sizes, NULL pointer, unknown enum); per chain:
                            a non-finite energy                                       */
    RGF_ENOMEM = 2,      /* device or host allocation failed                          */
    RGF_ECUDA = 3,       /* a CUDA runtime call failed                                */
    RGF_ENOCONV = 4,     /* lead decimation hit its iteration cap, went non-finite, or
                            missed the fixed point of the surface Dyson equation by
                            more than the residual tolerance (rgf_set_lead_controls)  */
    RGF_ESINGULAR = 5,   /* a zero pivot, or a pivot below 64 u max|A| (u the unit
                            roundoff of the working precision), in a slice inverse     */
    RGF_ENONFINITE = 6,  /* NaN or Inf in a slice Green's function or in T            */
    RGF_ETIMEOUT = 7,    /* a device-side wait exceeded its spin limit                */
    RGF_EBOUNDS = 8      /* T outside [0, n_ch(E)] (n_ch from the armchair band edges):
                            the sweep lost its accuracy at the working precision      */
} rgf_status;

typedef enum {
    RGF_FP64 = 0,        /* every step in IEEE binary64                               */
    RGF_MIXED = 1,       /* slice recursion in double-float (pairs of binary32 on the
                            FP32 pipes, ~48-bit significand); leads and trace binary64 */
    RGF_MIXED_TC = 2,    /* as RGF_MIXED, with the dense contractions of every slice
                            step (the rank-b updates of the slice inverse, the
                            corner-strip product of Eq. 5, the gradient's products) on
                            the tcgen05 tensor cores by exact bfloat16 digit slicing
                            of the double-float operands (see rgf_zgemm_tc)          */
    RGF_FP64_TC = 3      /* binary64 storage and ALU steps (as RGF_FP64), with the two
                            dense contractions of every slice step on the tensor cores,
                            sliced from binary64 and summed in binary64: products
                            accurate to a few units of 2^-53 of (row max x column max
                            x inner dimension), in the forward, gradient and LDOS
                            sweeps alike.
                            With both _TC precisions, ribbons wider than N = 1960
                            (ceil(N/2) > 980) run their products on the pipes, as
                            RGF_MIXED / RGF_FP64: the tensor-core tiles and the
                            sweep's panels no longer fit one block's shared memory. */
} rgf_precision;

/* One ribbon instance (the paper's input step: geometry, defects, disorder). */
typedef struct {
    int N;                     /* dimer lines, >= 2; orbitals per cell M = 2N          */
    int L;                     /* unit cells in the scattering region, >= 1            */
    double t;                  /* nearest-neighbour hopping in eV (e.g. -2.7)          */
    const double* onsite;      /* host [L][2N] on-site energies (eV), or NULL          */
    double anderson_W;         /* if onsite == NULL: eps ~ U[-W, W] from `seed`        */
    uint64_t seed;             /* SplitMix64 stream of the Anderson energies           */
    double edge_p;             /* if removed == NULL: rows 0 and N-1 atoms removed     */
    uint64_t edge_seed;        /*   with probability edge_p, from stream `edge_seed`   */
    const uint8_t* removed;    /* host [L][2N], 1 = atom absent, or NULL               */
} rgf_ribbon_desc;

typedef struct rgf_ribbon rgf_ribbon;   /* opaque; device-resident copy of a ribbon */

/*
 * Random inputs.  Draw i of stream s is the SplitMix64 output
 * mix64(s + (i+1) * 0x9E3779B97F4A7C15) and u = (bits >> 11) * 2^-53.
 * Orbital o of cell n uses draw n*2N + o.  Anderson: eps = W (2u - 1).
 * Edge roughness: an atom of row 0 or row N-1 is removed when u < p (other
 * rows are never drawn).  Leads are always pristine.
 *
 * rgf_generate_onsite: host only (no GPU needed).  Fills onsite_out[L*2N]
 * and removed_out[L*2N] (both host, caller-owned, either may be NULL) with
 * the arrays `desc` describes (copies when desc gives explicit arrays).
 * Errors: RGF_EINVAL.
 */
rgf_status rgf_generate_onsite(const rgf_ribbon_desc* desc, double* onsite_out,
                               uint8_t* removed_out);

/* Build a ribbon on the current device (generates or copies the arrays, then
 * uploads them).  *out is owned by the caller; release with rgf_free_ribbon.
 * Errors: RGF_EINVAL, RGF_ENOMEM, RGF_ECUDA. */
rgf_status rgf_build_ribbon(const rgf_ribbon_desc* desc, rgf_ribbon** out);

/* Same, from arrays already on the device: onsite_dev [L*2N] (binary64) and
 * removed_dev [L*2N] (uint8, or NULL for none).  The arrays are copied
 * device-to-device on `stream`; the caller may free them once the stream has
 * passed this call. */
rgf_status rgf_build_ribbon_dev(int N, int L, double t, const double* onsite_dev,
                                const uint8_t* removed_dev, void* stream, rgf_ribbon** out);

void rgf_free_ribbon(rgf_ribbon* rib);

/*
 * Lead self-energies by Lopez Sancho-Rubio decimation (binary64), one per
 * energy, for the pristine ribbon of N dimer lines (paper: the self-energies
 * of the leads enter at the first and the last slice, text after Eqs. 4-5).
 *   side 0: Sigma_L = H01^T g_s H01 on the first device cell (left lead);
 *   side 1: Sigma_R = H01 g_s H01^T on the last device cell (right lead);
 * with z = E + i*eta and the decimation stopped when the largest entry of the
 * effective couplings is below 1e-14 eV (cap 200 iterations by default).  The
 * pristine lead separates into transverse modes, and the decimation runs per
 * mode; each mode's surface Green's function g must then satisfy the surface
 * Dyson equation g = 1/(z - t^2/(z - tau^2 g)) to a relative residual of 1e-10
 * (by default; see rgf_set_lead_controls), else the energy fails.
 * sigma: host [nE][2N][2N] complex, interleaved (re, im) binary64, row-major
 *        (caller-owned, 8*nE*(2N)^2 doubles).
 * iters: host [nE] or NULL: iterations used, or -1 where decimation failed.
 * Returns RGF_ENOCONV if any energy failed (its sigma entries are NaN).
 */
rgf_status rgf_lead_selfenergy(int N, double t, const double* E, int nE, double eta,
                               int side, double* sigma, int* iters);

/*
 * Conductance T (in units of 2e^2/h) for `nchains` independent chains.  Chain c
 * is ribbon rib[c] at energy E[c] (several chains may share a ribbon).
 * eta_device is the broadening inside the scattering region, eta_lead the one
 * of the lead decimation.
 *
 * Method: the recursion of Eqs. 4-5 over the four atom columns of each unit
 * cell, run as two halves at the same time -- from the left lead up to the
 * middle of the ribbon and from the right lead down to it -- and joined by one
 * Dyson step (Eq. 3) across the middle bond; T = Tr[Gamma_L G_1L Gamma_R
 * G_1L^dagger] (Eq. 2) evaluated in the leads' transverse-mode bases.  The
 * lead-attached column at each end is formed and inverted in binary64 in the
 * mode basis of its lead, where the lead self-energy is diagonal, so that the
 * order-1/eta self-energies of the surface-state modes near E = 0 do not
 * swamp the order-1 terms (see rgf_lead_selfenergy); the join and the trace
 * are binary64; `precision` sets the arithmetic of the column recursion.
 *   rib:   host array of nchains ribbon pointers.
 *   E:     host [nchains] energies (eV).
 *   T:     host [nchains] output.
 *   chain_status: host [nchains] int32 output (rgf_status per chain) or NULL.
 * Errors: RGF_EINVAL, RGF_ENOMEM, RGF_ECUDA, or the first per-chain failure.
 */
rgf_status rgf_conductance(const rgf_ribbon* const* rib, const double* E, int nchains,
                           double eta_device, double eta_lead, int precision,
                           double* T, int32_t* chain_status);

/* Same with device buffers and a caller stream (E_dev, T_dev, status_dev on
 * the device; status_dev may be NULL).  Asynchronous: returns after launch;
 * results are valid once `stream` has passed the call.  Launch-time errors are
 * returned; per-chain failures appear in status_dev (a non-finite energy as
 * RGF_EINVAL). */
rgf_status rgf_conductance_dev(const rgf_ribbon* const* rib, const double* E_dev, int nchains,
                               double eta_device, double eta_lead, int precision,
                               void* stream, double* T_dev, int32_t* status_dev);

/*
 * Schedule of the forward sweep of rgf_conductance[_dev] (no counterpart in
 * the paper; process-wide, default RGF_SCHED_PHASED).  Both run the same
 * arithmetic in separately compiled kernels, so their T agree to rounding (the
 * compiler may fuse a product and a sum into one FMA in one of them only);
 * each is deterministic, whatever order the queue hands the work out in.
 *   RGF_SCHED_PHASED: three launches (end-column preparation, half sweeps,
 *     joins), blocks longest chain first; the hardware block scheduler hands
 *     each freed SM the next half.
 *   RGF_SCHED_PERSISTENT: after the lead decimation, one persistent kernel per
 *     launch group (one block per SM) takes the halves of the chains from a
 *     device work queue, longest chain first; the block that finishes the
 *     second half of a chain joins the two and writes T.  No block waits for
 *     another, so there is no queue wait that could time out.  It overlaps the
 *     preparations and joins with other chains' sweeps, but its recursion,
 *     compiled inside the queue loop beside the binary64 steps, runs about 7%
 *     slower on GB300 than the phased kernel's, hence the default.
 * A launch group is the set of chains on one engine: with RGF_MIXED_TC or
 * RGF_FP64_TC, the chains that the tuning table (rgf_set_tuning) sends to the
 * pipes run after the tensor-core group, as RGF_MIXED or RGF_FP64.  Errors:
 * RGF_EINVAL.
 */
typedef enum { RGF_SCHED_PERSISTENT = 0, RGF_SCHED_PHASED = 1 } rgf_schedule;
rgf_status rgf_set_schedule(int schedule);
int rgf_get_schedule(void);

/*
 * Domains per chain (no counterpart in the paper; process-wide; default 2,
 * 0 = automatic).  A chain's columns are cut into ndom domains that run at the
 * same time, one SM each: the two lead-attached halves at the ends and ndom - 2
 * interior domains between them, each recursed as a segment open at its first
 * column (an absorbing self-energy there, taken back out when it is joined)
 * that keeps the blocks of its first and last columns (G_aa, G_ab, g_b).  A
 * tree of joins (the Dyson equation across each boundary bond, binary64; in
 * the _TC precisions its products on the tensor cores, sliced from binary64)
 * combines the interior domains in ceil(log2(ndom - 2)) launches; the merge
 * then joins the left half, the combined interior and the right half.  This
 * is the modified recursion that running one chain in parallel needs: it
 * shortens a chain's sequential depth about ndom / 2 times, at one more
 * product per interior column step.
 * Automatic: as many domains as give every chain of the call one SM per domain
 * (2 while there are more than SMs / 2 chains, the bench batches), at most
 * ncol / 32 (ncol = 4 L of the shortest chain); rgf_auto_domains returns that
 * choice for nchains chains, a shortest chain of ncol_min columns and nsm SMs
 * (plain host call).  Forced values (>= 2) are capped at ncol / 2.  With more
 * than two domains the sweep runs the three-launch schedule.  Accuracy: each
 * join forms the Green's function of a grown segment at a free cut, which near
 * E = 0 is as ill-conditioned as the middle cut of the two halves, so the
 * rounding of the joins adds up: at L = 4000 (bench ribbon, 25 domains,
 * binary64) T stays within 3e-12 of 40-digit-pinned values away from E = 0
 * but moves to 2e-9 at |E| <= 5 meV (1e-10 with two domains); hence the
 * default of two.  The gradient and LDOS sweeps and rgf_conductance_noalloc
 * always use the two halves.  Errors: RGF_EINVAL (ndom not 0 and outside
 * [2, 4096]).
 */
rgf_status rgf_set_domains(int ndom);
int rgf_get_domains(void);
int rgf_auto_domains(int nchains, int ncol_min, int nsm);

/*
 * A prepared batch: the conductance of a fixed list of chains as one CUDA
 * graph (energies into the descriptors, lead decimation, then the sweep in the
 * schedule in force at creation: work-queue reset and persistent kernel, or
 * the three launches), built once and launched any number of times.
 * rgf_batch_create plans the chains (schedule from the tuning table in force),
 * allocates and uploads the batch's descriptors and workspace (cudaMalloc;
 * about the device memory of one rgf_conductance_dev call), and captures the
 * launches on a private stream.  The graph keeps the pointers it was created
 * with: every launch reads the energies in E_dev [nchains] and the ribbons'
 * on-site energies as they are when it runs, and writes T_dev [nchains] and
 * status_dev [nchains] (may be NULL); the caller keeps them, and the ribbons,
 * alive until rgf_batch_free.  The decimation controls (rgf_set_lead_controls)
 * are those in force at creation.  With profiling on at creation
 * (rgf_profile_enable) the graph records the profile events, and
 * rgf_profile_read_phases reads them after a launch.  rgf_batch_launch
 * enqueues the graph on `stream` and returns; launches of one batch share its
 * workspace and must not overlap (one stream, or events between streams).
 * Results equal those of rgf_conductance_dev under the same schedule bit for
 * bit.  Errors:
 * RGF_EINVAL (as rgf_conductance_dev; nchains must be >= 1), RGF_ENOMEM,
 * RGF_ECUDA (the capture or the launch failed).
 */
typedef struct rgf_batch rgf_batch;   /* opaque */
rgf_status rgf_batch_create(const rgf_ribbon* const* rib, const double* E_dev, int nchains,
                            double eta_device, double eta_lead, int precision, double* T_dev,
                            int32_t* status_dev, rgf_batch** out);
rgf_status rgf_batch_launch(rgf_batch* batch, void* stream);
void rgf_batch_free(rgf_batch* batch);

/*
 * Conductance and its gradient dT/d eps for every on-site energy of the
 * scattering region: dT/d eps_i = 2 Re (G_iL Gamma_R G_1L^dagger Gamma_L G_1i)
 * (from Eqs. 1-2), with the blocks of G assembled slice by slice through the
 * Dyson equation (Eq. 3) from the recursion of Eqs. 4-5 run from both leads.
 * The right-connected Green's functions are checkpointed every ckpt_stride
 * unit cells and recomputed between checkpoints; ckpt_stride <= 0 picks
 * ~sqrt(L).  Device workspace per chain: (14 + 2 ceil(4L / (4 s)) +
 * 2 (4 s + 1)) ceil(N/2)^2 complex values (s the stride), 16 bytes each.
 * T comes from this sweep's own left-to-right recursion with the lead
 * self-energies in the site basis; it agrees with rgf_conductance to the
 * working precision (not bit for bit), except near E = 0, where only
 * rgf_conductance treats the surface-state modes of the leads in their mode
 * basis.
 *   dT_deps: host [nchains][L*2N] binary64 (row-major per chain, orbital
 *            order of rgf_ribbon_desc); 0 on removed atoms.
 * Other arguments and errors as rgf_conductance.
 */
rgf_status rgf_conductance_grad(const rgf_ribbon* const* rib, const double* E, int nchains,
                                double eta_device, double eta_lead, int precision,
                                int ckpt_stride, double* T, double* dT_deps,
                                int32_t* chain_status);

/*
 * Same as rgf_conductance_grad with device buffers and a caller stream
 * (asynchronous: results are valid once `stream` has passed the call).
 * E_dev [nchains], T_dev [nchains], status_dev [nchains] (or NULL) on the device.
 *   weights_dev NULL:  dT_dev [nchains][L*2N] (device), per chain, packed in
 *                      chain order (chain c at the sum of the sizes before it);
 *   weights_dev [nchains] (device): dT_dev [L*2N] = sum_c weights[c] dT_c/d eps,
 *                      the vector-Jacobian product of the chains' T (every
 *                      ribbon must have the same N and L; summed over chains in
 *                      order, deterministic).  A failed chain contributes 0.
 * Launch-time errors are returned; per-chain failures appear in status_dev.
 */
rgf_status rgf_conductance_grad_dev(const rgf_ribbon* const* rib, const double* E_dev,
                                    int nchains, double eta_device, double eta_lead,
                                    int precision, int ckpt_stride, const double* weights_dev,
                                    void* stream, double* T_dev, double* dT_dev,
                                    int32_t* status_dev);

/*
 * Local density of states rho_i(E) = -Im G_ii(E) / pi (states per eV per
 * orbital) at every site of the scattering region.  The paper notes that the
 * Green's function of Eq. 1 gives every quantity of interest, the charge
 * density among them (text after Eq. 1); rho is that density's integrand over
 * energy.  The diagonal block G_kk of each column k comes from the Dyson
 * equation (Eq. 3) with the bonds on both sides of column k cut, joining the
 * recursion of Eqs. 4-5 run from the left lead with the same recursion run
 * from the right lead (checkpointed every ckpt_stride unit cells, as in
 * rgf_conductance_grad, with the same workspace).
 *   rho: host [nchains][L*2N] binary64 (row-major per chain, orbital order of
 *        rgf_ribbon_desc); 0 on removed atoms.
 *   T:   host [nchains], as rgf_conductance_grad returns it.
 * Other arguments and errors as rgf_conductance_grad.
 */
rgf_status rgf_ldos(const rgf_ribbon* const* rib, const double* E, int nchains,
                    double eta_device, double eta_lead, int precision, int ckpt_stride,
                    double* T, double* rho, int32_t* chain_status);

/*
 * Complex matrix product C = A B on the tcgen05 tensor cores: the dense
 * product the recursion forms at every slice (Eqs. 4-5; the paper's CGEMM
 * calls), here by exact bfloat16 digit slicing of the binary64 operands
 * (Ozaki scheme: 7 signed base-256 digits per real value from its
 * significand, per-row and per-column power-of-two scales), binary32
 * tensor-core accumulation that is exact for the five leading digit levels,
 * and binary64 recombination -- the product RGF_FP64_TC uses.  Accuracy per
 * entry: a few units of 2^-53 times k max_j |A_mj| max_j |B_jn| (at most
 * 2^-50 k max|A_m.| max|B_.n| per real part).
 *   A: device [m][lda], lda >= k;  B: device [k][ldb], ldb >= n;
 *   C: device [m][ldc], ldc >= n;  complex binary64, interleaved (re, im),
 *   row-major, leading dimensions in complex elements; C must not overlap
 *   A or B.  Inputs are caller-owned and unchanged.
 * Runs on `stream` and waits for it before returning.
 * Errors: RGF_EINVAL (negative size, short leading dimension, NULL pointer),
 * RGF_ECUDA, RGF_ETIMEOUT (a tensor-core completion wait gave up; C invalid).
 */
rgf_status rgf_zgemm_tc(int m, int n, int k, const double* A, int lda, const double* B, int ldb,
                        double* C, int ldc, void* stream);

/*
 * Self-test of the bounded tensor-core completion wait (no counterpart in the
 * paper).  Runs one 64 x 64 x 64 rgf_zgemm_tc product on the legacy default
 * stream with the MMA completion never committed to the mbarrier the kernel
 * waits on and a wait limit of about half a millisecond of device clock, so
 * that the wait runs out.  The kernel then sets its error flag, commits the
 * MMAs still in flight to a second mbarrier, waits for them (bounded), frees
 * its tensor memory and returns; the CUDA context stays usable.  Allocates and
 * frees its own 192 KiB device buffer.
 * Returns RGF_ETIMEOUT when the timeout path works; RGF_OK would mean that the
 * wait did not run out; RGF_ECUDA on a CUDA error.
 */
rgf_status rgf_zgemm_tc_selftest_timeout(void);

/*
 * Allocation-free variant of rgf_conductance_dev (no counterpart in the paper).
 *
 * For callers that may not allocate device memory: e.g. a host application
 * that has reserved the device memory for its own pool and forbids further
 * cudaMalloc, a plugin whose host only hands it pre-allocated buffers, or a
 * loop that must not trigger the implicit device synchronisation of
 * cudaMalloc / cudaFree.  This call performs no cudaMalloc, cudaFree or other
 * allocating call and copies nothing from host memory: its scratch (chain and
 * lead descriptors, lead workspace and output, sweep workspace) lives in one
 * fixed 64 MiB device array inside the library, which every GPU that loads
 * the library's device code holds until the process exits.  CUDA loads device
 * code lazily by default, so the array is created by the first call on each
 * device (or at context creation when CUDA_MODULE_LOADING=EAGER is set): a
 * caller that reserves the remaining device memory for itself should make one
 * call first.
 *
 * One ribbon of N dimer lines and L cells, given as device arrays
 * onsite_dev [L][2N] (binary64) and removed_dev [L][2N] (uint8, or NULL),
 * evaluated at nE energies E_dev [nE] (device).  Outputs on the device:
 * T_dev [nE], status_dev [nE] (int32, or NULL), as rgf_conductance_dev, in any
 * precision (RGF_FP64, RGF_MIXED, RGF_MIXED_TC, RGF_FP64_TC), by the three
 * launches of
 * RGF_SCHED_PHASED with the default schedule of every chain (the tuning table
 * is not read).  Asynchronous on `stream`; results are valid once the stream
 * has passed the call.  Returns RGF_EINVAL,
 * with a message naming the limit, when the scratch the call needs exceeds
 * 64 MiB (21 energies at N = 245, more at smaller N); split the energies over
 * several calls then.
 *
 * The array is shared by all calls and keeps the last call's contents; two
 * calls whose GPU work overlaps (different streams, or a second call before
 * the first has finished) race on it.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress) and caches it; make that
 * first call before any stream capture.  After cudaDeviceReset of a device the
 * cached address is stale: do not use this entry point on that device again in
 * the same process.
 */
rgf_status rgf_conductance_noalloc(int N, int L, double t, const double* onsite_dev,
                                   const uint8_t* removed_dev, const double* E_dev, int nE,
                                   double eta_device, double eta_lead, int precision,
                                   void* stream, double* T_dev, int32_t* status_dev);

/*
 * Diagnostics (no counterpart in the paper).  When enabled, every
 * rgf_conductance* call records CUDA events on its stream around its two
 * kernel phases: lead decimation and slice sweep (with the trace).
 * rgf_profile_read waits for the last call's events and returns the phase
 * durations in milliseconds (either pointer may be NULL).  Process-wide
 * state: not for concurrent calls from several threads.  Errors: RGF_ECUDA,
 * RGF_EINVAL if profiling is off or no call was recorded.
 */
rgf_status rgf_profile_enable(int on);
rgf_status rgf_profile_read(double* ms_lead, double* ms_sweep);

/* The phases of the last profiled rgf_conductance* call, in milliseconds:
 * ms[0] lead decimation, ms[1] end-column preparation, ms[2] half sweeps (the
 * gradient sweep for rgf_conductance_grad), ms[3] join and trace.  Under
 * RGF_SCHED_PERSISTENT the preparation and the join run inside the persistent
 * kernel: ms[2] is that kernel (all launch groups), ms[1] the work-queue reset
 * and ms[3] zero.  rgf_profile_read's ms_sweep is ms[1] + ms[2] + ms[3].
 * ms: host [4]. */
rgf_status rgf_profile_read_phases(double* ms);

/*
 * Decimation controls (no counterpart in the paper; process-wide, for
 * diagnostics and host-side fault injection): the iteration cap of every mode
 * (default 200) and the relative residual tolerance of the surface Dyson
 * equation (default 1e-10) that rgf_lead_selfenergy and every rgf_conductance*
 * call apply.  A cap of 1, or a tolerance of 0, makes the energies fail with
 * RGF_ENOCONV without any device fault.  Errors: RGF_EINVAL (max_iter outside
 * [1, 100000], residual_tol negative or NaN).
 */
rgf_status rgf_set_lead_controls(int max_iter, double residual_tol);

/*
 * Tuning of the forward sweep per column size (no counterpart in the paper;
 * process-wide, one table per precision).  Entry i applies to the chains whose
 * column size K = ceil(N/2) is at most K_max[i] and above K_max[i-1]; chains
 * wider than the last entry take the last entry; with no table every chain
 * takes the default {engine RGF_ENGINE_TENSOR, panel 0, pairs 1}.
 *   engine: RGF_ENGINE_TENSOR (the dense products on the tcgen05 tensor cores)
 *           or RGF_ENGINE_PIPES (on the FP32 / FP64 pipes); only RGF_MIXED_TC
 *           and RGF_FP64_TC read it.
 *   panel:  Gauss-Jordan panel width 2, 4, 8 or 16, capped by the shared memory
 *           of the launch; 0 = the widest that fits.
 *   pairs:  1 = t I-bonded column pairs share one inverse (where no atom of the
 *           second column is within 1e-4 eV of resonance), 0 = one column at a
 *           time.
 * Every schedule computes the same recursion; results differ only by rounding.
 * rgf_set_tuning installs a table of n <= RGF_TUNE_MAX_ENTRIES entries with
 * K_max strictly increasing (n = 0 removes it); rgf_get_tuning copies the
 * installed table (*n its length; RGF_EINVAL if cap is smaller);
 * rgf_tune_lookup returns the entry a ribbon of width N gets.  Plain host
 * calls (no device needed).  Errors: RGF_EINVAL.
 *
 * rgf_autotune measures, for each width N[i], one Anderson-disordered chain
 * (W = 0.1 eV) of `cells` unit cells at E = 0.3 eV under every candidate --
 * engine (both with the _TC precisions) x panel {16, 8, 4} x pairs {1, 0}, *ncand
 * of them -- as the device time of its half sweeps (the middle launch of
 * RGF_SCHED_PHASED, CUDA events; the minimum of `reps` runs after one
 * warm-up), writes
 * the fastest into best[i] (K_max = ceil(N[i]/2)) and the times into ms
 * [nN][*ncand] (may be NULL), and installs the table.  The widths must have
 * distinct column sizes.  Synchronous; uses the current device.  Errors:
 * RGF_EINVAL, RGF_ENOMEM, RGF_ECUDA.
 */
#define RGF_TUNE_MAX_ENTRIES 64
#define RGF_TUNE_MAX_CANDIDATES 12
typedef enum { RGF_ENGINE_PIPES = 0, RGF_ENGINE_TENSOR = 1 } rgf_engine;
typedef struct {
    int K_max;
    int engine;
    int panel;
    int pairs;
} rgf_tune_entry;
rgf_status rgf_set_tuning(int precision, const rgf_tune_entry* table, int n);
rgf_status rgf_get_tuning(int precision, rgf_tune_entry* table, int cap, int* n);
rgf_status rgf_tune_lookup(int precision, int N, rgf_tune_entry* out);
rgf_status rgf_autotune(int precision, const int* N, int nN, int cells, int reps,
                        rgf_tune_entry* best, double* ms, int* ncand);

const char* rgf_status_str(int status);
const char* rgf_last_error(void);

/* Library version string. */
const char* rgf_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RGF_H */
