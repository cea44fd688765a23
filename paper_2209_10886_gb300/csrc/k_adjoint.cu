// Adjoint-state gradient of the source-receiver misfit
//     J = 1/2 sum_s || P u_s - d_s ||^2,   A(m2) u_s = h^2 f_s.
// A is complex symmetric and depends on m2 only through its diagonal:
//     dA_pp/dm2_p = -omega^2 h^2 - n_outer(p) (2/(1-beta_p)^2) (i omega h / (4 sqrt(m2_p))),
//     beta_p = i omega h sqrt(m2_p) / 2.
// With L_s = A^{-1} conj(P^T (P u_s - d_s)) (= conj(lambda_s)):
//     grad_p = - sum_s Re( L_{s,p} dA_pp/dm2_p u_{s,p} ).
#include "helm_internal.cuh"

namespace {

__global__ void receiver_residual_kernel(const double2* __restrict__ u, long long N, const int* __restrict__ rec, int nrec,
                                         const double2* __restrict__ d, double2* __restrict__ res,
                                         double* __restrict__ partial) {
    __shared__ double sh[256];
    const int s = blockIdx.x;
    double acc = 0.0;
    for (int k = threadIdx.x; k < nrec; k += blockDim.x) {
        const double2 uv = HLD(u + (long long)s * N + HLD(rec + k));
        const double2 dv = HLD(d + (long long)s * nrec + k);
        const double2 rv = make_double2(uv.x - dv.x, uv.y - dv.y);
        HST(res + (long long)s * nrec + k, rv);
        acc += rv.x * rv.x + rv.y * rv.y;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[s] = 0.5 * sh[0];
}

// f_adj_s = conj(P^T res_s) / h^2  (so that A x = h^2 f_adj is the adjoint system)
__global__ void adjoint_rhs_kernel(const double2* __restrict__ res, const int* __restrict__ rec, int nrec, long long N,
                                   double inv_h2, double2* __restrict__ f_adj) {
    const int s = blockIdx.x;
    if (threadIdx.x != 0) return;     // serial per source: receivers may repeat
    for (int k = 0; k < nrec; ++k) {
        const double2 rv = HLD(res + (long long)s * nrec + k);
        double2* t = f_adj + (long long)s * N + HLD(rec + k);
        if (!HELM_CHK(t, sizeof(double2))) continue;
        t->x += rv.x * inv_h2;
        t->y += -rv.y * inv_h2;
    }
}

__global__ void gradient_kernel(const double2* __restrict__ U, const double2* __restrict__ Lt, const double* __restrict__ m2,
                                int nx, int ny, double h, double omega, int nsrc, double* __restrict__ grad) {
    const long long N = (long long)nx * ny;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < N; p += (long long)gridDim.x * blockDim.x) {
        const int a = (int)(p % nx), b = (int)(p / nx);
        const int nouter = (a == 0) + (a == nx - 1) + (b == 0) + (b == ny - 1);
        const double m = HLD(m2 + p);
        const double wh = omega * h;
        double2 da = make_double2(-wh * wh, 0.0);
        if (nouter) {
            const double2 one_m = make_double2(1.0, -0.5 * wh * sqrt(m));             // 1 - beta
            const double2 sq = make_double2(one_m.x * one_m.x - one_m.y * one_m.y, 2.0 * one_m.x * one_m.y);
            const double2 dc = cdiv(make_double2(2.0, 0.0), sq);                       // 2/(1-beta)^2
            const double db = wh / (4.0 * sqrt(m));                                    // dbeta/dm2 = i db
            da.x -= nouter * (-dc.y * db);
            da.y -= nouter * (dc.x * db);
        }
        double g = 0.0;
        for (int s = 0; s < nsrc; ++s) {
            const double2 l = HLD(Lt + (long long)s * N + p), u = HLD(U + (long long)s * N + p);
            const double2 lu = make_double2(l.x * u.x - l.y * u.y, l.x * u.y + l.y * u.x);
            g -= lu.x * da.x - lu.y * da.y;
        }
        HST(grad + p, g);
    }
}

}  // namespace

void launch_receiver_residual(const double2* u, long long N, const int* rec, int nrec, const double2* d, int nsrc,
                              double2* res, double* partial, cudaStream_t st) {
    count_launch();
    receiver_residual_kernel<<<nsrc, 256, 0, st>>>(u, N, rec, nrec, d, res, partial);
}
void launch_adjoint_rhs(const double2* res, const int* rec, int nrec, int nsrc, long long N, double inv_h2,
                        double2* f_adj, cudaStream_t st) {
    count_launch();
    adjoint_rhs_kernel<<<nsrc, 32, 0, st>>>(res, rec, nrec, N, inv_h2, f_adj);
}
void launch_gradient(const double2* U, const double2* Lt, const double* m2, int nx, int ny, double h, double omega,
                     int nsrc, double* grad, cudaStream_t st) {
    long long N = (long long)nx * ny;
    int nb = (int)min((N + 255) / 256, (long long)152 * 8);
    count_launch();
    gradient_kernel<<<nb, 256, 0, st>>>(U, Lt, m2, nx, ny, h, omega, nsrc, grad);
}
