// rgf_lead.cu -- semi-infinite lead self-energies by Lopez Sancho-Rubio
// decimation, binary64, one thread block per (energy, side).
//
// The paper includes the lead self-energies at the first and last slice (text
// after Eqs. 4-5).  Decimation (Lopez Sancho, Lopez Sancho, Rubio 1985) on a
// principal layer of one unit cell iterates
//     g = (z - eps)^-1;  eps_s += a g b;  eps += a g b + b g a;
//     a <- a g a;  b <- b g b
// until the effective coupling a (and b = a^T) vanishes, then
// g_s = (z - eps_s)^-1.  In the column slicing of a cell (columns c0..c3 at
// x = 0, a, 1.5a, 2.5a) the cell-to-cell hopping only joins column c3 of one
// cell to column c0 of the next, so every correction lives on the c0c0 and
// c3c3 blocks and a on the c3->c0 (or c0->c3) block.  Each iteration only needs
// the four corner blocks of (z - eps)^-1 on {c0, c3}; they come from a left
// and a right sweep through the cell's four columns.  Same algebra as the
// full-cell iteration, on KL x KL / KR x KR blocks instead of 2N x 2N.
//   right lead: a0 = H(c3 -> c0'), corrections of eps_s on c3, g_s needed on c0,
//               Sigma_R = W30 g_s[c0c0] W30^T  (acts on c3 of the last cell)
//   left lead:  a0 = H(c0 -> c3'), corrections of eps_s on c0, g_s needed on c3,
//               Sigma_L = W30^T g_s[c3c3] W30  (acts on c0 of the first cell)
#include "rgf_device.cuh"
#include "rgf_internal.h"

namespace rgf {

size_t sweep_smem_bytes(int Kmax);

namespace {

struct LeadSmem {
    GJSmem<double> gj;
    zd* gemm;
    double* red;
};

__device__ LeadSmem carve_lead(unsigned char* base, int Kmax) {
    LeadSmem s;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + o;
        o += (bytes + 15) & ~(size_t)15;
        return p;
    };
    s.gj.rowbuf = (zd*)take((size_t)Kmax * 16);
    s.gj.colbuf = (zd*)take((size_t)Kmax * 16);
    s.gj.colval = (zd*)take((size_t)Kmax * 16);
    s.gemm = (zd*)take(2 * 8 * 64 * 16);
    s.gj.inv = (zd*)take(16);
    s.gj.colabs = (double*)take((size_t)Kmax * 8);
    take((size_t)Kmax * 8);
    s.red = (double*)take(NWARP * 8);
    s.gj.perm = (int*)take((size_t)Kmax * 4);
    s.gj.idx = (int*)take((size_t)Kmax * 4);
    s.gj.ctl = (int*)take(16);
    return s;
}

// X (K x K, ld) = z I - D - s * Y   (D, Y may be null)
__device__ void shift_minus(zd* X, int K, int ld, zd z, const zd* D, const zd* Y, double s) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < K; i += NWARP)
        for (int l = lane; l < K; l += 32) {
            zd v = (i == l) ? z : zd{0.0, 0.0};
            if (D) v = csub(v, D[(size_t)i * ld + l]);
            if (Y) v = csub(v, cscale(Y[(size_t)i * ld + l], s));
            X[(size_t)i * ld + l] = v;
        }
    __syncthreads();
}

// X (KR x KR) = z I - t^2 * [sum over p in {q,q+1}, p' in {q',q'+1}] F[p][p']
// (W12^T F W12 with F of size KL).
__device__ void x_from_w12T_F_w12(zd* X, int KL, int KR, int ld, zd z, const zd* F, double t2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int q = warp; q < KR; q += NWARP)
        for (int r = lane; r < KR; r += 32) {
            zd s = {0.0, 0.0};
            for (int a = q; a <= q + 1; ++a)
                for (int b = r; b <= r + 1; ++b)
                    if (a < KL && b < KL) s = cadd(s, F[(size_t)a * ld + b]);
            zd v = (q == r) ? z : zd{0.0, 0.0};
            X[(size_t)q * ld + r] = csub(v, cscale(s, t2));
        }
    __syncthreads();
}

// X (KL x KL) = z I - t^2 * [sum over q in {p-1,p}, q' in {p'-1,p'}] F[q][q']
// (W12 F W12^T with F of size KR).
__device__ void x_from_w12_F_w12T(zd* X, int KL, int KR, int ld, zd z, const zd* F, double t2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = warp; p < KL; p += NWARP)
        for (int r = lane; r < KL; r += 32) {
            zd s = {0.0, 0.0};
            for (int a = p - 1; a <= p; ++a)
                for (int b = r - 1; b <= r; ++b)
                    if (a >= 0 && b >= 0 && a < KR && b < KR) s = cadd(s, F[(size_t)a * ld + b]);
            zd v = (p == r) ? z : zd{0.0, 0.0};
            X[(size_t)p * ld + r] = csub(v, cscale(s, t2));
        }
    __syncthreads();
}

__device__ void addto2(zd* A, zd* B, const zd* S, int m, int n, int ld) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = warp; i < m; i += NWARP)
        for (int l = lane; l < n; l += 32) {
            zd v = S[(size_t)i * ld + l];
            A[(size_t)i * ld + l] = cadd(A[(size_t)i * ld + l], v);
            if (B) B[(size_t)i * ld + l] = cadd(B[(size_t)i * ld + l], v);
        }
    __syncthreads();
}

__device__ void zero(zd* A, int m, int n, int ld) {
    for (int e = threadIdx.x; e < m * n; e += NT) A[(size_t)(e / n) * ld + (e % n)] = {0.0, 0.0};
    __syncthreads();
}

}  // namespace

__global__ void __launch_bounds__(NT, 1)
lead_kernel(const LeadDev* __restrict__ leads, int nlead, int Kmax, double eta,
            zd* __restrict__ ws, zd* __restrict__ out, int* __restrict__ lead_status,
            int* __restrict__ lead_iters) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LeadSmem s = carve_lead(smem_raw, Kmax);
    const int prob = blockIdx.x >> 1, side = blockIdx.x & 1;
    const LeadDev ld = leads[prob];
    const int N = ld.N, KL = col_KL(N), KR = col_KR(N), L2 = KL;   // ld of every block = KL
    const double t = ld.t, t2 = t * t;
    const zd z = {ld.E, eta};
    const size_t B = (size_t)KL * KL;
    zd* base = ws + ld.ws_off;
    zd *Xw = base, *f0 = base + B, *f1 = base + 2 * B, *f2 = base + 3 * B, *G33 = base + 4 * B;
    zd *r3 = base + 5 * B, *r2 = base + 6 * B, *r1 = base + 7 * B, *G00 = base + 8 * B;
    zd *G03 = base + 9 * B, *T1 = base + 10 * B, *T2 = base + 11 * B, *T3 = base + 12 * B;
    zd *a = base + 13 * B, *tmp = base + 14 * B, *tmp2 = base + 15 * B, *anew = base + 16 * B;
    zd *D0 = base + 17 * B, *D3 = base + 18 * B, *Ds = base + 19 * B;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    // a0: right lead KR x KL, a[q][p] = t for p in {q, q+1};
    //     left lead  KL x KR, a[p][q] = t for q in {p-1, p}.
    const int am = side ? KR : KL, an = side ? KL : KR;
    for (int e = threadIdx.x; e < am * an; e += NT) {
        int i = e / an, j = e % an;
        bool on = side ? (j == i || j == i + 1) : (j == i - 1 || j == i);
        a[(size_t)i * L2 + j] = on ? zd{t, 0.0} : zd{0.0, 0.0};
    }
    zero(D0, KL, KL, L2);
    zero(D3, KR, KR, L2);
    zero(Ds, side ? KR : KL, side ? KR : KL, L2);

    const double tol = 1e-14;
    const int max_iter = 200;
    int it = 0, ok = 0, flag = 0;
    for (it = 1; it <= max_iter; ++it) {
        // forward through c0..c3: G33 and G03
        shift_minus(Xw, KL, L2, z, D0, nullptr, 0.0);
        flag |= cta_gj_invert<double>(Xw, KL, L2, f0, L2, s.gj);
        shift_minus(Xw, KL, L2, z, nullptr, f0, t2);
        flag |= cta_gj_invert<double>(Xw, KL, L2, f1, L2, s.gj);
        x_from_w12T_F_w12(Xw, KL, KR, L2, z, f1, t2);
        flag |= cta_gj_invert<double>(Xw, KR, L2, f2, L2, s.gj);
        shift_minus(Xw, KR, L2, z, D3, f2, t2);
        flag |= cta_gj_invert<double>(Xw, KR, L2, G33, L2, s.gj);
        cta_gemm<double, false, false>(KL, KL, KL, f0, L2, f1, L2, T1, L2, GEMM_SET, s.gemm);
        for (int p = warp; p < KL; p += NWARP)
            for (int q = lane; q < KR; q += 32) {
                zd v = T1[(size_t)p * L2 + q];
                if (q + 1 < KL) v = cadd(v, T1[(size_t)p * L2 + q + 1]);
                T2[(size_t)p * L2 + q] = cscale(v, t2 * t);
            }
        __syncthreads();
        cta_gemm<double, false, false>(KL, KR, KR, T2, L2, f2, L2, T3, L2, GEMM_SET, s.gemm);
        cta_gemm<double, false, false>(KL, KR, KR, T3, L2, G33, L2, G03, L2, GEMM_SET, s.gemm);
        // backward through c3..c0: G00
        shift_minus(Xw, KR, L2, z, D3, nullptr, 0.0);
        flag |= cta_gj_invert<double>(Xw, KR, L2, r3, L2, s.gj);
        shift_minus(Xw, KR, L2, z, nullptr, r3, t2);
        flag |= cta_gj_invert<double>(Xw, KR, L2, r2, L2, s.gj);
        x_from_w12_F_w12T(Xw, KL, KR, L2, z, r2, t2);
        flag |= cta_gj_invert<double>(Xw, KL, L2, r1, L2, s.gj);
        shift_minus(Xw, KL, L2, z, D0, r1, t2);
        flag |= cta_gj_invert<double>(Xw, KL, L2, G00, L2, s.gj);

        if (side) {
            // a: KR x KL.  a g[c0c0] a^T -> c3c3 (eps and eps_s); a^T g[c3c3] a -> c0c0;
            // a <- a g[c0c3] a.
            cta_gemm<double, false, false>(KR, KL, KL, a, L2, G00, L2, tmp, L2, GEMM_SET, s.gemm);
            cta_gemm<double, false, true>(KR, KR, KL, tmp, L2, a, L2, tmp2, L2, GEMM_SET, s.gemm);
            addto2(D3, Ds, tmp2, KR, KR, L2);
            cta_gemm<double, true, false>(KL, KR, KR, a, L2, G33, L2, tmp, L2, GEMM_SET, s.gemm);
            cta_gemm<double, false, false>(KL, KL, KR, tmp, L2, a, L2, tmp2, L2, GEMM_SET, s.gemm);
            addto2(D0, nullptr, tmp2, KL, KL, L2);
            cta_gemm<double, false, false>(KR, KR, KL, a, L2, G03, L2, tmp, L2, GEMM_SET, s.gemm);
            cta_gemm<double, false, false>(KR, KL, KR, tmp, L2, a, L2, anew, L2, GEMM_SET, s.gemm);
        } else {
            // a: KL x KR.  a g[c3c3] a^T -> c0c0 (eps and eps_s); a^T g[c0c0] a -> c3c3;
            // a <- a g[c3c0] a = a G03^T a.
            cta_gemm<double, false, false>(KL, KR, KR, a, L2, G33, L2, tmp, L2, GEMM_SET, s.gemm);
            cta_gemm<double, false, true>(KL, KL, KR, tmp, L2, a, L2, tmp2, L2, GEMM_SET, s.gemm);
            addto2(D0, Ds, tmp2, KL, KL, L2);
            cta_gemm<double, true, false>(KR, KL, KL, a, L2, G00, L2, tmp, L2, GEMM_SET, s.gemm);
            cta_gemm<double, false, false>(KR, KR, KL, tmp, L2, a, L2, tmp2, L2, GEMM_SET, s.gemm);
            addto2(D3, nullptr, tmp2, KR, KR, L2);
            cta_gemm<double, false, true>(KL, KL, KR, a, L2, G03, L2, tmp, L2, GEMM_SET, s.gemm);
            cta_gemm<double, false, false>(KL, KR, KL, tmp, L2, a, L2, anew, L2, GEMM_SET, s.gemm);
        }
        double mx = 0.0;
        for (int e = threadIdx.x; e < am * an; e += NT) {
            size_t o = (size_t)(e / an) * L2 + (e % an);
            zd v = anew[o];
            a[o] = v;
            double m2 = cabs2(v);
            mx = (isnan(m2) || m2 > mx) ? m2 : mx;
        }
        mx = block_max(mx, s.red);
        if (!isfinite(mx) || (flag & 2)) break;
        if (mx < tol * tol) { ok = 1; break; }
    }

    zd* sig = out + ld.off + (side ? (size_t)KL * KL : 0);
    zd* gam = out + ld.off + (size_t)KL * KL + (size_t)KR * KR + (side ? (size_t)KL * KL : 0);
    const int K = side ? KR : KL;
    if (ok) {
        zd* gs;
        if (side) {
            // g_s on c0 of the surface cell; eps_s corrected on c3.
            shift_minus(Xw, KR, L2, z, Ds, nullptr, 0.0);
            flag |= cta_gj_invert<double>(Xw, KR, L2, r3, L2, s.gj);
            shift_minus(Xw, KR, L2, z, nullptr, r3, t2);
            flag |= cta_gj_invert<double>(Xw, KR, L2, r2, L2, s.gj);
            x_from_w12_F_w12T(Xw, KL, KR, L2, z, r2, t2);
            flag |= cta_gj_invert<double>(Xw, KL, L2, r1, L2, s.gj);
            shift_minus(Xw, KL, L2, z, nullptr, r1, t2);
            flag |= cta_gj_invert<double>(Xw, KL, L2, G00, L2, s.gj);
            gs = G00;
            // Sigma_R[q][q'] = t^2 sum_{p in {q,q+1}, p' in {q',q'+1}} gs[p][p']
            for (int q = warp; q < KR; q += NWARP)
                for (int r = lane; r < KR; r += 32) {
                    zd v = {0.0, 0.0};
                    for (int pa = q; pa <= q + 1; ++pa)
                        for (int pb = r; pb <= r + 1; ++pb)
                            if (pa < KL && pb < KL) v = cadd(v, gs[(size_t)pa * L2 + pb]);
                    sig[(size_t)q * KR + r] = cscale(v, t2);
                }
        } else {
            // g_s on c3 of the surface cell; eps_s corrected on c0.
            shift_minus(Xw, KL, L2, z, Ds, nullptr, 0.0);
            flag |= cta_gj_invert<double>(Xw, KL, L2, f0, L2, s.gj);
            shift_minus(Xw, KL, L2, z, nullptr, f0, t2);
            flag |= cta_gj_invert<double>(Xw, KL, L2, f1, L2, s.gj);
            x_from_w12T_F_w12(Xw, KL, KR, L2, z, f1, t2);
            flag |= cta_gj_invert<double>(Xw, KR, L2, f2, L2, s.gj);
            shift_minus(Xw, KR, L2, z, nullptr, f2, t2);
            flag |= cta_gj_invert<double>(Xw, KR, L2, G33, L2, s.gj);
            gs = G33;
            // Sigma_L[p][p'] = t^2 sum_{q in {p-1,p}, q' in {p'-1,p'}} gs[q][q']
            for (int p = warp; p < KL; p += NWARP)
                for (int r = lane; r < KL; r += 32) {
                    zd v = {0.0, 0.0};
                    for (int qa = p - 1; qa <= p; ++qa)
                        for (int qb = r - 1; qb <= r; ++qb)
                            if (qa >= 0 && qb >= 0 && qa < KR && qb < KR)
                                v = cadd(v, gs[(size_t)qa * L2 + qb]);
                    sig[(size_t)p * KL + r] = cscale(v, t2);
                }
        }
        __syncthreads();
        double bad = 0.0;
        for (int e = threadIdx.x; e < K * K; e += NT) {
            int i = e / K, j = e % K;
            zd sij = sig[(size_t)i * K + j], sji = sig[(size_t)j * K + i];
            // Gamma = i (Sigma - Sigma^dagger)
            double dr = sij.re - sji.re, di = sij.im + sji.im;
            gam[(size_t)i * K + j] = {-di, dr};
            if (!cfinite(sij)) bad = 1.0;
        }
        bad = block_max(bad, s.red);
        if (bad > 0.0 || (flag & 2)) ok = 0;
    }
    if (!ok) {
        for (int e = threadIdx.x; e < K * K; e += NT) {
            sig[e] = {NAN, NAN};
            gam[e] = {NAN, NAN};
        }
    }
    if (threadIdx.x == 0) {
        lead_status[2 * prob + side] = ok ? ST_OK : ST_ENOCONV;
        if (lead_iters) lead_iters[2 * prob + side] = ok ? it : -1;
    }
}

cudaError_t launch_lead(const LeadDev* leads, int nlead, int Kmax, double eta_lead, void* ws,
                        void* out, int* lead_status, int* lead_iters, cudaStream_t st) {
    if (nlead <= 0) return cudaSuccess;
    size_t smem = sweep_smem_bytes(Kmax);
    cudaError_t e = cudaFuncSetAttribute(lead_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    lead_kernel<<<2 * nlead, NT, smem, st>>>(leads, nlead, Kmax, eta_lead, (zd*)ws, (zd*)out,
                                             lead_status, lead_iters);
    return cudaGetLastError();
}

}  // namespace rgf
