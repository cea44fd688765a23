// Coefficient tables of the discretisation and of the Robin transmission
// (paper Eq. origPbm with T = i kappa on the outer boundary; Eq. subPbm on
// the interfaces).  All arithmetic in FP64; run once per helm_setup.
#include "helm_internal.cuh"

namespace {

__device__ double2 ghost_coef(double2 beta) {               // (1 + beta)/(1 - beta)
    return cdiv(make_double2(1.0 + beta.x, beta.y), make_double2(1.0 - beta.x, -beta.y));
}

// beta_e = T_e h / 2 for the interface edge with wavenumber kappa_e
__device__ double2 edge_beta(double kappa_e, double h, int transmission, double tc_scale) {
    if (transmission == HELM_TC_IMPEDANCE) return make_double2(0.0, 0.5 * kappa_e * h);
    const double p0 = tc_scale * sqrt(0.5 * kappa_e * 3.14159265358979323846 / h);
    return make_double2(-0.5 * p0 * h, 0.5 * p0 * h);          // T_e = (i - 1) p0
}

__device__ int find_cut(const int* cut, int nparts, int v) {    // part index k with cut[k] <= v < cut[k+1]
    int lo = 0, hi = nparts - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (cut[mid] <= v) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void setup_coeffs_kernel(const double* __restrict__ m2, int nx, int ny, double h, double omega,
                                    const int* __restrict__ xcut, const int* __restrict__ ycut, int N1, int N2,
                                    const int* __restrict__ subid, int transmission, double tc_scale,
                                    double2* __restrict__ adiag, double2* __restrict__ dloc,
                                    const SubDev* __restrict__ subtab) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)nx * ny) return;
    const int a = (int)(p % nx), b = (int)(p / nx);
    const double m = m2[p];
    const double kap = omega * sqrt(m);
    const double kh2 = kap * kap * h * h;
    const double2 cp = ghost_coef(make_double2(0.0, 0.5 * kap * h));
    const int nouter = (a == 0) + (a == nx - 1) + (b == 0) + (b == ny - 1);
    adiag[p] = make_double2(4.0 - kh2 - nouter * cp.x, -nouter * cp.y);

    const int i1 = find_cut(xcut, N1, a), i2 = find_cut(ycut, N2, b);
    const SubDev sd = subtab[subid[i2 * N1 + i1]];
    double2 d = make_double2(4.0 - kh2, 0.0);
    // the four sides of the node that leave its subdomain box
    const int on_side[4] = {a == sd.x0, a == sd.x0 + sd.mx - 1, b == sd.y0, b == sd.y0 + sd.my - 1};
    const int qa[4] = {a - 1, a + 1, a, a};
    const int qb[4] = {b, b, b - 1, b + 1};
    for (int s = 0; s < 4; ++s) {
        if (!on_side[s]) continue;
        double2 c;
        if (qa[s] < 0 || qa[s] >= nx || qb[s] < 0 || qb[s] >= ny) {
            c = cp;                                             // outer boundary: T = i kappa_p
        } else {
            const double mq = m2[(long long)qb[s] * nx + qa[s]];
            const double kap_e = omega * sqrt(0.5 * (m + mq));
            c = ghost_coef(edge_beta(kap_e, h, transmission, tc_scale));
        }
        d.x -= c.x;
        d.y -= c.y;
    }
    dloc[sd.loff + (long long)(b - sd.y0) * sd.mx + (a - sd.x0)] = d;
}

__global__ void trace_coeffs_kernel(const double* __restrict__ m2, int nx, double h, double omega,
                                    int transmission, double tc_scale, const int* __restrict__ slot_sub,
                                    const int* __restrict__ slot_side, const int* __restrict__ slot_off,
                                    const int* __restrict__ slot_len, const SubDev* __restrict__ subtab,
                                    TraceCoef<double2>* __restrict__ tc128, TraceCoef<float2>* __restrict__ tc64) {
    const int slot = blockIdx.x;
    const SubDev sd = subtab[slot_sub[slot]];
    const int side = slot_side[slot], off = slot_off[slot], len = slot_len[slot];
    for (int k = threadIdx.x; k < len; k += blockDim.x) {
        int ap, bp, aq, bq;
        if (side == SW || side == SE) {
            bp = bq = sd.y0 + k;
            ap = side == SW ? sd.x0 : sd.x0 + sd.mx - 1;
            aq = side == SW ? ap - 1 : ap + 1;
        } else {
            ap = aq = sd.x0 + k;
            bp = side == SS ? sd.y0 : sd.y0 + sd.my - 1;
            bq = side == SS ? bp - 1 : bp + 1;
        }
        const double mp = m2[(long long)bp * nx + ap], mq = m2[(long long)bq * nx + aq];
        const double2 beta = edge_beta(omega * sqrt(0.5 * (mp + mq)), h, transmission, tc_scale);
        const double2 one_m = make_double2(1.0 - beta.x, -beta.y);
        const double2 cin = cdiv(make_double2(1.0, 0.0), one_m);
        const double2 ca = cdiv(make_double2(-(1.0 + beta.x), -beta.y), one_m);
        const double2 cb = cdiv(make_double2(-4.0 * beta.x, -4.0 * beta.y), one_m);
        TraceCoef<double2> t128{cin, ca, cb};
        tc128[off + k] = t128;
        TraceCoef<float2> t64{to_c64(cin), to_c64(ca), to_c64(cb)};
        tc64[off + k] = t64;
    }
}

}  // namespace

void launch_setup_coeffs(const double* m2, int nx, int ny, double h, double omega, const int* xcut,
                         const int* ycut, int N1, int N2, const int* subid, int transmission, double tc_scale,
                         double2* adiag, double2* dloc, const SubDev* subtab, cudaStream_t st) {
    long long N = (long long)nx * ny;
    int nb = (int)((N + 255) / 256);
    count_launch();
    setup_coeffs_kernel<<<nb, 256, 0, st>>>(m2, nx, ny, h, omega, xcut, ycut, N1, N2, subid, transmission,
                                             tc_scale, adiag, dloc, subtab);
}

void launch_trace_coeffs(const double* m2, int nx, double h, double omega, int transmission, double tc_scale,
                         const int* slot_sub, const int* slot_side, const int* slot_off, const int* slot_len,
                         int nslots, const SubDev* subtab, TraceCoef<double2>* tc128, TraceCoef<float2>* tc64,
                         cudaStream_t st) {
    if (nslots == 0) return;
    count_launch();
    trace_coeffs_kernel<<<nslots, 128, 0, st>>>(m2, nx, h, omega, transmission, tc_scale, slot_sub, slot_side,
                                                slot_off, slot_len, subtab, tc128, tc64);
}
