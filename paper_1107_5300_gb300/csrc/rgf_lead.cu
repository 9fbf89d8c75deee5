// rgf_lead.cu -- semi-infinite lead self-energies by Lopez Sancho-Rubio
// decimation, binary64, one thread block per energy (both leads).
//
// The paper includes the lead self-energies at the first and last slice (text
// after Eqs. 4-5).  The leads are pristine armchair ribbons, so the lead
// Hamiltonian separates exactly into transverse modes: with
// phi_p(j) = sin(p pi (j+1)/(N+1)) on rows j = 0..N-1, the vector
// phi_p restricted to the even rows (columns c0, c1 of a cell) is mapped by the
// row +-1 hopping stencil onto 2 cos(p pi/(N+1)) times phi_p restricted to the
// odd rows (columns c2, c3), because phi_p(j-1) + phi_p(j+1) = 2 cos(...) phi_p(j)
// and phi_p vanishes at j = -1 and j = N.  Modes p = 1..KL are an orthogonal
// basis of the even rows, p = 1..KR of the odd rows.  Each mode is a chain
//     c0 -t- c1 -tau- c2 -t- c3 -tau- c0' -t- ...,   tau_p = 2 t cos(p pi/(N+1)),
// i.e. a two-site principal layer (A -t- B) joined by tau.  Sancho-Rubio
// decimation of that layer,
//     g = (z - eps)^-1;  eps_s += a g b;  eps += a g b + b g a;  a <- a g a; b <- b g b
// keeps a on the B->A' entry, the corrections on the A and B diagonal, and
// stops when |a| < 1e-14 eV.  The surface Green's function at the first atom of
// a semi-infinite mode chain (for both leads the outermost bond is t) is
//     g_p = (z - s_B) / (z (z - s_B) - t^2).
// Back in real space, with u_p the normalised restricted mode vectors:
//     Sigma_L = sum_p tau_p^2 g_p u_p^even u_p^even^T   (on c0 of the first cell)
//     Sigma_R = sum_p tau_p^2 g_p u_p^odd  u_p^odd^T    (on c3 of the last cell)
// which equal H01^T g_s H01 and H01 g_s H01^T of the full-cell iteration, at
// O(N) work per iteration instead of O(N^3) and without inverting isolated
// sub-blocks of the cell.  The output also carries the mode vectors and the
// mode self-energies w_p = tau_p^2 g_p themselves: the sweep works on the
// lead-attached columns in the mode basis, where Sigma is diagonal (near
// E = 0 the surface-state modes have |w_p| ~ 1/eta).
//
// Checks: a non-finite energy is RGF_EINVAL; a mode that reaches the iteration
// cap, goes non-finite, or whose g_p misses the fixed point of the surface
// Dyson equation g = 1/(z - t^2/(z - tau^2 g)) by more than the residual
// tolerance (relative) is RGF_ENOCONV.
#include "rgf_device.cuh"
#include "rgf_internal.h"

namespace rgf {

namespace {

constexpr double kTol = 1e-14;

LeadControls g_controls = {200, 1e-10};

// Mode p (1-based) of an N-line ribbon: surface Green's function and iterations.
__device__ zd mode_surface(int p, int N, double t, zd z, int max_iter, int& iters, bool& ok) {
    const double tau = 2.0 * t * cospi((double)p / (double)(N + 1));
    zd a = {tau, 0.0};
    zd dA = {0.0, 0.0}, dB = {0.0, 0.0}, sB = {0.0, 0.0};
    const zd tt = {t * t, 0.0};
    ok = false;
    int it;
    for (it = 1; it <= max_iter; ++it) {
        zd zA = csub(z, dA), zB = csub(z, dB);
        zd det = csub(cmul(zA, zB), tt);
        double d2 = det.re * det.re + det.im * det.im;
        zd idet = {det.re / d2, -det.im / d2};
        zd gAA = cmul(zB, idet), gBB = cmul(zA, idet), gAB = cscale(idet, t);
        zd a2 = cmul(a, a);
        zd agb = cmul(a2, gAA), bga = cmul(a2, gBB);
        dB = cadd(dB, agb);
        sB = cadd(sB, agb);
        dA = cadd(dA, bga);
        a = cmul(a2, gAB);
        double ma = a.re * a.re + a.im * a.im;
        if (!isfinite(ma) || !cfinite(dA) || !cfinite(dB)) break;
        if (ma < kTol * kTol) { ok = true; break; }
    }
    iters = it;
    zd zs = csub(z, sB);
    zd den = csub(cmul(z, zs), tt);
    double d2 = den.re * den.re + den.im * den.im;
    zd g = cmul(zs, zd{den.re / d2, -den.im / d2});
    if (!cfinite(g)) ok = false;
    return g;
}

// Relative residual |g - 1/(z - t^2/(z - tau^2 g))| / |g| of the surface Dyson
// equation of mode chain p (bonds t, tau, t, ... from the surface atom).
__device__ double mode_residual(zd g, double t, double tau, zd z) {
    const zd inner = csub(z, cscale(g, tau * tau));
    const zd t2i = cscale(crecip(inner), t * t);
    const zd rhs = crecip(csub(z, t2i));
    const zd d = csub(g, rhs);
    return sqrt((d.re * d.re + d.im * d.im) / (g.re * g.re + g.im * g.im));
}

// Normalised restricted mode vectors: U[i][p-1] = phi_p(row of entry i) / norm,
// rows 2i + parity, i < K.  sinpi with an exactly reduced argument.
__device__ void mode_basis(double* U, int K, int N, int parity, double* red) {
    const int twoN2 = 2 * (N + 1);
    for (int e = threadIdx.x; e < K * K; e += NT) {
        int i = e / K, p = e % K + 1;
        long long m = ((long long)(2 * i + parity + 1) * p) % twoN2;
        U[e] = sinpi((double)m / (double)(N + 1));
    }
    __syncthreads();
    // column norms
    for (int p = threadIdx.x; p < K; p += NT) {
        double s = 0.0;
        for (int i = 0; i < K; ++i) s += U[i * K + p] * U[i * K + p];
        red[p] = rsqrt(s);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += NT) U[e] *= red[e % K];
    __syncthreads();
}

// S[i][j] = sum_p U[i][p] w[p] U[j][p];  Gam = i (S - S^dagger).
__device__ void assemble(zd* S, zd* Gam, const double* U, const zd* w, int K) {
    for (int e = threadIdx.x; e < K * K; e += NT) {
        int i = e / K, j = e % K;
        double re = 0.0, im = 0.0;
        for (int p = 0; p < K; ++p) {
            double u = U[i * K + p] * U[j * K + p];
            re = fma(u, w[p].re, re);
            im = fma(u, w[p].im, im);
        }
        S[e] = {re, im};
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * K; e += NT) {
        int i = e / K, j = e % K;
        zd sij = S[(size_t)i * K + j], sji = S[(size_t)j * K + i];
        double dr = sij.re - sji.re, di = sij.im + sji.im;
        Gam[e] = {-di, dr};
    }
    __syncthreads();
}

}  // namespace

LeadControls lead_controls() { return g_controls; }
void set_lead_controls(LeadControls c) { g_controls = c; }

__global__ void __launch_bounds__(NT, 1)
lead_kernel(const LeadDev* __restrict__ leads, int nlead, double eta, int max_iter,
            double residual_tol, double* __restrict__ ws, zd* __restrict__ out,
            int* __restrict__ lead_status, int* __restrict__ lead_iters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int prob = blockIdx.x;
    const LeadDev ld = leads[prob];
    const int N = ld.N, KL = col_KL(N), KR = col_KR(N);
    zd* w = reinterpret_cast<zd*>(smem_raw);                    // [KL]
    double* red = reinterpret_cast<double*>(w + KL);             // [max(KL, NWARP)]
    int* flags = reinterpret_cast<int*>(red + (KL > NWARP ? KL : NWARP));   // [2]
    if (threadIdx.x == 0) { flags[0] = 1; flags[1] = 0; }
    __syncthreads();
    const zd z = {ld.E, eta};
    const bool finite_E = isfinite(ld.E);
    for (int p = threadIdx.x; p < KL && finite_E; p += NT) {
        int it;
        bool ok;
        zd g = mode_surface(p + 1, N, ld.t, z, max_iter, it, ok);
        const double tau = 2.0 * ld.t * cospi((double)(p + 1) / (double)(N + 1));
        if (ok && !(mode_residual(g, ld.t, tau, z) <= residual_tol)) ok = false;
        w[p] = cscale(g, tau * tau);
        if (!ok) atomicExch(&flags[0], 0);
        atomicMax(&flags[1], it);
    }
    __syncthreads();
    const bool ok = finite_E && flags[0] != 0;
    zd* SigL = out + ld.off;
    zd* SigR = SigL + (size_t)KL * KL;
    zd* GamL = SigR + (size_t)KR * KR;
    zd* GamR = GamL + (size_t)KL * KL;
    zd* UL = GamR + (size_t)KR * KR;
    zd* UR = UL + (size_t)KL * KL;
    zd* wout = UR + (size_t)KR * KR;
    double* U = ws + 2 * ld.ws_off;
    if (ok) {
        mode_basis(U, KL, N, 0, red);
        assemble(SigL, GamL, U, w, KL);
        for (int e = threadIdx.x; e < KL * KL; e += NT) UL[e] = {U[e], 0.0};
        __syncthreads();
        mode_basis(U, KR, N, 1, red);
        assemble(SigR, GamR, U, w, KR);
        for (int e = threadIdx.x; e < KR * KR; e += NT) UR[e] = {U[e], 0.0};
        for (int p = threadIdx.x; p < KL; p += NT) wout[p] = w[p];
    } else {
        for (int e = threadIdx.x; e < KL * KL; e += NT) SigL[e] = GamL[e] = UL[e] = {NAN, NAN};
        for (int e = threadIdx.x; e < KR * KR; e += NT) SigR[e] = GamR[e] = UR[e] = {NAN, NAN};
        for (int p = threadIdx.x; p < KL; p += NT) wout[p] = {NAN, NAN};
    }
    if (threadIdx.x == 0) {
        const int st = ok ? ST_OK : (finite_E ? ST_ENOCONV : ST_EINVAL);
        lead_status[2 * prob] = lead_status[2 * prob + 1] = st;
        if (lead_iters) lead_iters[2 * prob] = lead_iters[2 * prob + 1] = ok ? flags[1] : -1;
    }
}

cudaError_t launch_lead(const LeadDev* leads, int nlead, int Kmax, double eta_lead, void* ws,
                        void* out, int* lead_status, int* lead_iters, cudaStream_t st) {
    if (nlead <= 0) return cudaSuccess;
    size_t smem = (size_t)Kmax * 16 + (size_t)(Kmax > NWARP ? Kmax : NWARP) * 8 + 16;
    const LeadControls ctl = lead_controls();
    lead_kernel<<<nlead, NT, smem, st>>>(leads, nlead, eta_lead, ctl.max_iter, ctl.residual_tol,
                                         (double*)ws, (zd*)out, lead_status, lead_iters);
    return cudaGetLastError();
}

}  // namespace rgf
