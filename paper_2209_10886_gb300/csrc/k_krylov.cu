// FP64 kernels of the flexible GMRES solver (paper Section 6: GMRES to a
// relative residual of 1e-6) and of the five-point operator.
//
// Reductions are deterministic: every block writes its partial sums, a second
// kernel adds them in a fixed order.
#include "helm_internal.cuh"

#include <algorithm>

namespace {

constexpr int NTH = 256;

template <typename V> __device__ __forceinline__ V warp_sum(V v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// block-wide sum of one double; result valid in thread 0
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// (A u)_p = adiag_p u_p - sum_{grid neighbours} u_q     (h^2-scaled five-point operator)
__device__ __forceinline__ double2 apply_A(const double2* __restrict__ u, const double2 ad, long long p, int a, int b,
                                           int nx, int ny) {
    double sx = 0.0, sy = 0.0;
    if (a > 0) { double2 q = HLD(u + p - 1); sx += q.x; sy += q.y; }
    if (a < nx - 1) { double2 q = HLD(u + p + 1); sx += q.x; sy += q.y; }
    if (b > 0) { double2 q = HLD(u + p - nx); sx += q.x; sy += q.y; }
    if (b < ny - 1) { double2 q = HLD(u + p + nx); sx += q.x; sy += q.y; }
    const double2 c = HLD(u + p);
    return make_double2(fma(ad.x, c.x, fma(-ad.y, c.y, -sx)), fma(ad.x, c.y, fma(ad.y, c.x, -sy)));
}

// grid: x covers a row of the grid in NTH-wide segments, y strides over rows, z = RHS
__global__ void matvec_kernel(const double2* __restrict__ adiag, int nx, int ny, const double2* __restrict__ u,
                              double2* __restrict__ Au) {
    const long long N = (long long)nx * ny;
    const int k = blockIdx.z;
    const int a = blockIdx.x * NTH + threadIdx.x;
    if (a >= nx) return;
    const double2* uk = u + k * N;
    for (int b = blockIdx.y; b < ny; b += gridDim.y) {
        const long long p = (long long)b * nx + a;
        HST(Au + k * N + p, apply_A(uk, HLD(adiag + p), p, a, b, nx, ny));
    }
}

// r = fscale f - A u, and per-block partial ||r||^2 (partial index: y * gridDim.x + x)
__global__ void residual_kernel(const double2* __restrict__ adiag, int nx, int ny, const double2* __restrict__ f,
                                double fscale, const double2* __restrict__ u, double2* __restrict__ r,
                                const int* __restrict__ active, double* __restrict__ partial) {
    __shared__ double sh[32];
    const long long N = (long long)nx * ny;
    const int k = blockIdx.z;
    const int nb = gridDim.x * gridDim.y, bid = blockIdx.y * gridDim.x + blockIdx.x;
    if (active && !active[k]) {
        if (threadIdx.x == 0) partial[(long long)k * nb + bid] = 0.0;
        return;
    }
    const int a = blockIdx.x * NTH + threadIdx.x;
    const double2* uk = u + k * N;
    double acc = 0.0;
    if (a < nx) {
        for (int b = blockIdx.y; b < ny; b += gridDim.y) {
            const long long p = (long long)b * nx + a;
            const double2 Av = apply_A(uk, HLD(adiag + p), p, a, b, nx, ny);
            const double2 fv = HLD(f + k * N + p);
            const double2 rv = make_double2(fma(fscale, fv.x, -Av.x), fma(fscale, fv.y, -Av.y));
            HST(r + k * N + p, rv);
            acc = fma(rv.x, rv.x, fma(rv.y, rv.y, acc));
        }
    }
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) HST(partial + (long long)k * nb + bid, acc);
}

template <typename VT>
__global__ void norm2_partial_kernel(const VT* __restrict__ v, long long n, long long stride,
                                     double* __restrict__ partial) {
    using Re = decltype(VT::x);
    __shared__ double sh[32];
    const int k = blockIdx.y;
    Re acc = 0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const VT x = HLD(v + k * stride + p);
        acc = fma(x.x, x.x, fma(x.y, x.y, acc));
    }
    const double t = block_sum((double)acc, sh);
    if (threadIdx.x == 0) HST(partial + (long long)k * gridDim.x + blockIdx.x, t);
}

// out[row] = sum_b partial[row][b]   (mode 1: sqrt of the sum)
__global__ void reduce_rows_kernel(const double* __restrict__ partial, int nblk, double* __restrict__ out, int mode) {
    __shared__ double sh[32];
    const int row = blockIdx.x;
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) acc += HLD(partial + (long long)row * nblk + b);
    acc = block_sum(acc, sh);
    if (threadIdx.x == 0) HST(out + row, mode == 1 ? sqrt(acc) : acc);
}

// partial[k][blk][j] = sum_{p in block range} conj(V_j[p]) w[p],  j < nvec (summed in the
// vectors' precision within a block, in FP64 across blocks)
constexpr int KB = 4;
template <typename VT>
__global__ void mdot_kernel(const VT* __restrict__ V, long long vsk, long long vsr, int nvec,
                            const VT* __restrict__ w, long long ws, long long n, const int* __restrict__ active,
                            double2* __restrict__ partial) {
    __shared__ double sh[32];
    const int k = blockIdx.y;
    const int nblk = gridDim.x;
    double2* out = partial + ((long long)k * nblk + blockIdx.x) * nvec;
    if (active && !active[k]) {
        for (int j = threadIdx.x; j < nvec; j += blockDim.x) out[j] = make_double2(0.0, 0.0);
        return;
    }
    const long long chunk = (n + nblk - 1) / nblk;
    const long long p0 = blockIdx.x * chunk, p1 = min(n, p0 + chunk);
    const VT* wk = w + k * ws;
    for (int j0 = 0; j0 < nvec; j0 += KB) {
        VT acc[KB];
#pragma unroll
        for (int q = 0; q < KB; ++q) acc[q] = czero<VT>();
        for (long long p = p0 + threadIdx.x; p < p1; p += blockDim.x) {
            const VT wv = HLD(wk + p);
#pragma unroll
            for (int q = 0; q < KB; ++q)
                if (j0 + q < nvec) acc[q] = cfmaconj(HLD(V + (long long)(j0 + q) * vsk + k * vsr + p), wv, acc[q]);
        }
#pragma unroll
        for (int q = 0; q < KB; ++q) {
            if (j0 + q >= nvec) break;
            const double re = block_sum((double)acc[q].x, sh);
            const double im = block_sum((double)acc[q].y, sh);
            if (threadIdx.x == 0) HST(out + j0 + q, make_double2(re, im));
        }
    }
}

__global__ void reduce_cpartials_kernel(const double2* __restrict__ partial, int nblk, int nvec,
                                        double2* __restrict__ out, long long os) {
    __shared__ double sh[32];
    const int k = blockIdx.y, j = blockIdx.x;
    double re = 0.0, im = 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
        const double2 v = HLD(partial + ((long long)k * nblk + b) * nvec + j);
        re += v.x;
        im += v.y;
    }
    re = block_sum(re, sh);
    im = block_sum(im, sh);
    if (threadIdx.x == 0) HST(out + k * os + j, make_double2(re, im));
}

// w += sign * sum_j coef[k][j] V_j, optional per-block ||w||^2 partials (the update in
// the vectors' precision with the FP64 coefficients rounded to it)
template <typename VT>
__global__ void mupdate_kernel(const VT* __restrict__ V, long long vsk, long long vsr, int nvec,
                               const int* __restrict__ nvec_rhs, const double2* __restrict__ coef, long long cs,
                               double sign, VT* __restrict__ w, long long ws, long long n,
                               const int* __restrict__ active, double* __restrict__ norm_partial) {
    using Re = decltype(VT::x);
    __shared__ VT c[512];
    __shared__ double sh[32];
    const int k = blockIdx.y;
    const bool on = !(active && !active[k]);
    const int nv = nvec_rhs ? nvec_rhs[k] : nvec;
    for (int j = threadIdx.x; j < nv && j < 512; j += blockDim.x) {
        const double2 cj = coef[k * cs + j];
        c[j] = mk((Re)(sign * cj.x), (Re)(sign * cj.y));
    }
    __syncthreads();
    Re acc = 0;
    if (on) {
        VT* wk = w + k * ws;
        for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
            VT x = HLD(wk + p);
            for (int j = 0; j < nv; ++j) x = cfma(c[j], HLD(V + (long long)j * vsk + k * vsr + p), x);
            HST(wk + p, x);
            acc = fma(x.x, x.x, fma(x.y, x.y, acc));
        }
    }
    if (norm_partial) {
        const double t = block_sum((double)acc, sh);
        if (threadIdx.x == 0) norm_partial[(long long)k * gridDim.x + blockIdx.x] = t;
    }
}

// dst = src * inv[k]  (inactive RHS: dst = 0)
template <typename VT>
__global__ void scale_vec_kernel(VT* __restrict__ dst, long long ds, const VT* __restrict__ src,
                                 long long ss, const double* __restrict__ inv, long long n,
                                 const int* __restrict__ active) {
    using Re = decltype(VT::x);
    const int k = blockIdx.y;
    const bool on = !(active && !active[k]);
    const Re s = on ? (Re)inv[k] : (Re)0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const VT x = on ? HLD(src + k * ss + p) : czero<VT>();
        HST(dst + k * ds + p, mk(x.x * s, x.y * s));
    }
}

// One Arnoldi column j per RHS: H(0..j, j) = h1 + h2, H(j+1, j) = ||w||, then the
// Givens rotations of the earlier columns, a new rotation that annihilates
// H(j+1, j), and the rotated right-hand side g.  |g_{j+1}| is the residual norm
// of the least-squares problem min ||beta e_1 - H y||.
// one warp per RHS: the column and the earlier rotations are gathered into shared
// memory by all lanes, lane 0 runs the serial chain of rotations there
__global__ void hessenberg_step_kernel(double2* __restrict__ H, int ldh, long long hs, double2* __restrict__ cs,
                                       double2* __restrict__ sn, double2* __restrict__ g, int ldg,
                                       const double2* __restrict__ hcol, long long hcs, const double* __restrict__ hnorm,
                                       int j, int nrhs, const int* __restrict__ active,
                                       double* __restrict__ resid_est, double* __restrict__ inv_hnext) {
    extern __shared__ double2 hsm[];                 // col[j+2], cs[j+1], sn[j+1]
    const int k = blockIdx.x, lane = threadIdx.x;
    if (k >= nrhs || (active && !active[k])) return;
    double2* col = hsm;
    double2* csv = col + (j + 2);
    double2* snv = csv + (j + 1);
    double2* csk = cs + (long long)k * ldg;
    double2* snk = sn + (long long)k * ldg;
    const double hn = hnorm[k];
    for (int i = lane; i <= j; i += 32) {
        col[i] = hcol[k * hcs + i];
        if (i < j) { csv[i] = csk[i]; snv[i] = snk[i]; }
    }
    __syncwarp();
    if (lane == 0) {
        col[j + 1] = make_double2(hn, 0.0);
        double2* gk = g + (long long)k * ldg;
        double2 gj = gk[j], gj1;
        givens_column<double2>(col, csv, snv, j, gj, gj1);
        gk[j] = gj;
        gk[j + 1] = gj1;
        csk[j] = csv[j];
        snk[j] = snv[j];
        resid_est[k] = sqrt(gj1.x * gj1.x + gj1.y * gj1.y);
        inv_hnext[k] = hn > 0.0 ? 1.0 / hn : 0.0;
    }
    __syncwarp();
    double2* colg = H + k * hs + (long long)j * ldh;       // column-major: H(i, jj) at H[jj*ldh + i]
    for (int i = lane; i <= j + 1; i += 32) HST(colg + i, col[i]);
}

// y = R^{-1} g (upper triangular R = rotated H, first jcount[k] columns)
// one warp per RHS: the right-hand side (and, for up to HS_SMEM columns, the upper
// triangle of R) in shared memory, then column-oriented back substitution: y_i from
// row i, every lane subtracts R(r, i) y_i from its rows r < i
constexpr int HS_SMEM = 48;
__global__ void hessenberg_solve_kernel(const double2* __restrict__ H, int ldh, long long hs, const double2* __restrict__ g,
                                        int ldg, const int* __restrict__ jcount, double2* __restrict__ y, int ldy, int nrhs,
                                        bool cache_ok) {
    // rhs[m] | R[m][m] (column-major; allocated only when the restart length is at most HS_SMEM)
    extern __shared__ double2 hsm2[];
    const int k = blockIdx.x, lane = threadIdx.x;
    if (k >= nrhs) return;
    const int m = jcount[k];
    const double2* Hk = H + k * hs;
    double2* yk = y + (long long)k * ldy;
    double2* rhs = hsm2;
    double2* R = hsm2 + m;
    const bool cached = cache_ok && m <= HS_SMEM;
    for (int i = lane; i < m; i += 32) rhs[i] = HLD(g + (long long)k * ldg + i);
    if (cached)
        for (int c = 0; c < m; ++c)
            for (int r = lane; r <= c; r += 32) R[c * m + r] = HLD(Hk + (long long)c * ldh + r);
    __syncwarp();
    for (int i = m - 1; i >= 0; --i) {
        const double2 d = cached ? R[i * m + i] : HLD(Hk + (long long)i * ldh + i);
        const double2 yi = cdiv(rhs[i], d);
        if (lane == 0) HST(yk + i, yi);
        for (int r = lane; r < i; r += 32) {
            const double2 h = cached ? R[i * m + r] : HLD(Hk + (long long)i * ldh + r);
            double2 v = rhs[r];
            v.x -= h.x * yi.x - h.y * yi.y;
            v.y -= h.x * yi.y + h.y * yi.x;
            rhs[r] = v;
        }
        __syncwarp();
    }
}

__global__ void sqrt_kernel(double* v, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = sqrt(v[i]);
}

// norm -> (1/norm, norm) with zero norms mapped to (1, 1)
__global__ void scale_from_norm_kernel(const double* norm2, double* inv, double* scale, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = sqrt(norm2[i]);
    inv[i] = s > 0.0 ? 1.0 / s : 1.0;
    scale[i] = s > 0.0 ? s : 1.0;
}

int grid_for(long long n) {
    long long b = (n + NTH - 1) / NTH;
    return (int)min(b, (long long)152 * 8);
}

}  // namespace

static dim3 rows_grid(int nx, int ny, int nblk, int nrhs) {
    const int gx = (nx + NTH - 1) / NTH;
    const int gy = max(1, min(ny, nblk / gx));
    return dim3(gx, gy, nrhs);
}
void launch_matvec(const double2* adiag, int nx, int ny, const double2* u, double2* Au, int nrhs, cudaStream_t st) {
    count_launch();
    matvec_kernel<<<rows_grid(nx, ny, 152 * 16, nrhs), NTH, 0, st>>>(adiag, nx, ny, u, Au);
}
// returns the number of partials per RHS written into `partial` (<= nblk)
int launch_residual(const double2* adiag, int nx, int ny, const double2* f, double fscale, const double2* u,
                    double2* r, int nrhs, const int* active, double* partial, int nblk, cudaStream_t st) {
    const dim3 g = rows_grid(nx, ny, nblk, nrhs);
    count_launch();
    residual_kernel<<<g, NTH, 0, st>>>(adiag, nx, ny, f, fscale, u, r, active, partial);
    return (int)(g.x * g.y);
}
template <typename VT>
void launch_norm2_partial(const VT* v, long long n, int nrhs, long long stride, double* partial, int nblk,
                          cudaStream_t st) {
    dim3 g(nblk, nrhs);
    count_launch();
    norm2_partial_kernel<VT><<<g, NTH, 0, st>>>(v, n, stride, partial);
}
void launch_reduce_rows(const double* partial, int nblk, int nrows, double* out, int mode, cudaStream_t st) {
    count_launch();
    reduce_rows_kernel<<<nrows, NTH, 0, st>>>(partial, nblk, out, mode);
}
template <typename VT>
void launch_mdot(const VT* V, long long vsk, long long vsr, int nvec, const VT* w, long long ws, long long n,
                 int nrhs, const int* active, double2* partial, int nblk, cudaStream_t st) {
    dim3 g(nblk, nrhs);
    count_launch();
    mdot_kernel<VT><<<g, NTH, 0, st>>>(V, vsk, vsr, nvec, w, ws, n, active, partial);
}
void launch_reduce_cpartials(const double2* partial, int nblk, int nrows, double2* out, long long os, int nrhs,
                             cudaStream_t st) {
    dim3 g(nrows, nrhs);
    count_launch();
    reduce_cpartials_kernel<<<g, NTH, 0, st>>>(partial, nblk, nrows, out, os);
}
template <typename VT>
void launch_mupdate(const VT* V, long long vsk, long long vsr, int nvec, const int* nvec_rhs, const double2* coef,
                    long long cs, double sign, VT* w, long long ws, long long n, int nrhs, const int* active,
                    double* norm_partial, int nblk, cudaStream_t st) {
    dim3 g(nblk, nrhs);
    count_launch();
    mupdate_kernel<VT><<<g, NTH, 0, st>>>(V, vsk, vsr, nvec, nvec_rhs, coef, cs, sign, w, ws, n, active,
                                                 norm_partial);
}
template <typename VT>
void launch_scale_vec(VT* dst, long long ds, const VT* src, long long ss, const double* inv, long long n,
                      int nrhs, const int* active, cudaStream_t st) {
    dim3 g(grid_for(n), nrhs);
    count_launch();
    scale_vec_kernel<VT><<<g, NTH, 0, st>>>(dst, ds, src, ss, inv, n, active);
}
#define HELM_VEC_INST(VT)                                                                                          \
    template void launch_norm2_partial<VT>(const VT*, long long, int, long long, double*, int, cudaStream_t);       \
    template void launch_mdot<VT>(const VT*, long long, long long, int, const VT*, long long, long long, int,       \
                                  const int*, double2*, int, cudaStream_t);                                         \
    template void launch_mupdate<VT>(const VT*, long long, long long, int, const int*, const double2*, long long,   \
                                     double, VT*, long long, long long, int, const int*, double*, int,              \
                                     cudaStream_t);                                                                 \
    template void launch_scale_vec<VT>(VT*, long long, const VT*, long long, const double*, long long, int,        \
                                       const int*, cudaStream_t);
HELM_VEC_INST(double2)
HELM_VEC_INST(float2)
#undef HELM_VEC_INST
void launch_hessenberg_step(double2* H, int ldh, long long hs, double2* cs, double2* sn, double2* g, int ldg,
                            const double2* hcol, long long hcs, const double* hnorm, int j, int nrhs, const int* active,
                            double* resid_est, double* inv_hnext, cudaStream_t st) {
    count_launch();
    hessenberg_step_kernel<<<nrhs, 32, (size_t)(3 * j + 4) * sizeof(double2), st>>>(
        H, ldh, hs, cs, sn, g, ldg, hcol, hcs, hnorm, j, nrhs, active, resid_est, inv_hnext);
}
void launch_hessenberg_solve(const double2* H, int ldh, long long hs, const double2* g, int ldg, const int* jcount,
                             double2* y, int ldy, int nrhs, cudaStream_t st) {
    count_launch();
    // shared memory for the largest possible m (the restart length, at most ldh - 1)
    const int mmax = ldh - 1;
    const size_t smem = (size_t)(mmax + (mmax <= HS_SMEM ? mmax * mmax : 0)) * sizeof(double2);
    hessenberg_solve_kernel<<<nrhs, 32, smem, st>>>(H, ldh, hs, g, ldg, jcount, y, ldy, nrhs, mmax <= HS_SMEM);
}
void launch_sqrt_inplace(double* v, int n, cudaStream_t st) {
    count_launch();
    sqrt_kernel<<<(n + 127) / 128, 128, 0, st>>>(v, n);
}
void launch_scale_from_norm(const double* norm2, double* inv, double* scale, int n, cudaStream_t st) {
    count_launch();
    scale_from_norm_kernel<<<(n + 127) / 128, 128, 0, st>>>(norm2, inv, scale, n);
}

// ------------------------------------------------------- c128 -> c64 scaling
__global__ void to_c64_scaled_kernel(const double2* __restrict__ src, const double* __restrict__ scale,
                                     float2* __restrict__ out, long long n, int nrhs) {
    const long long total = n * nrhs;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const double sc = HLD(scale + i / n);
        const double2 v = HLD(src + i);
        HST(out + i, make_float2((float)(v.x * sc), (float)(v.y * sc)));
    }
}

void launch_to_c64_scaled(const double2* src, const double* scale, float2* out, long long n, int nrhs,
                          cudaStream_t st) {
    count_launch();
    to_c64_scaled_kernel<<<1216, 256, 0, st>>>(src, scale, out, n, nrhs);
}

// ------------------------------------------------- interface (trace) vectors
// T: the trace buffers' complex type (the factors' precision); VT: the interface
// Krylov vectors' type.  Same types: plain copies and sums in that precision.
template <typename O, typename I> __device__ __forceinline__ O cvt(I a);
template <> __device__ __forceinline__ float2 cvt<float2, float2>(float2 a) { return a; }
template <> __device__ __forceinline__ double2 cvt<double2, double2>(double2 a) { return a; }
template <> __device__ __forceinline__ double2 cvt<double2, float2>(float2 a) { return to_c128(a); }
template <> __device__ __forceinline__ float2 cvt<float2, double2>(double2 a) { return to_c64(a); }

// out = sign * (a + b) for n * nrhs values, b optional; with dj, out is the Krylov slot
// *dj + joff of an array of slots vsk apart (the slot index read on the device)
// (and into out2, optional, unshifted: may be a, each element is read before it is written)
// (launched with a programmatic dependency: waits for the previous kernel before any
// access, lets the next one launch at once)
template <typename T, typename VT>
__global__ void trace_to_kernel(const T* a, const T* __restrict__ b, int sign, VT* __restrict__ out,
                                long long total, const int* dj, int joff, long long vsk, VT* out2) {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    if (dj) out += (long long)(*dj + joff) * vsk;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        VT v = cvt<VT>(HLD(a + i));
        if (b) v = cadd(v, cvt<VT>(HLD(b + i)));
        if (sign < 0) v = mk(-v.x, -v.y);
        HST(out + i, v);
        if (out2) HST(out2 + i, v);
    }
}
// out (and out2, optional) = in rounded to T; with dj, in is the slot *dj + joff
template <typename VT, typename T>
__global__ void trace_from_kernel(const VT* __restrict__ in, T* __restrict__ out, T* __restrict__ out2,
                                  long long total, const int* dj, int joff, long long vsk) {
    if (dj) in += (long long)(*dj + joff) * vsk;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const T f = cvt<T>(HLD(in + i));
        HST(out + i, f);
        if (out2) HST(out2 + i, f);
    }
}
// r = b - w
template <typename VT>
__global__ void sub_kernel(const VT* __restrict__ b, const VT* __restrict__ w, VT* __restrict__ r, long long total) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x)
        HST(r + i, csub(HLD(b + i), HLD(w + i)));
}

static int small_grid(long long total) { return (int)std::min<long long>(1216, (total + 255) / 256 + 1); }

// launch of kernel `k` with a programmatic dependency on the previous kernel of the stream
template <typename... P, typename... A>
static cudaError_t launch_pdl(void (*k)(P...), dim3 grid, dim3 block, cudaStream_t st, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

template <typename T, typename VT>
void launch_trace_to(const T* a, const T* b, int sign, VT* out, long long total, cudaStream_t st, const int* dj,
                     int joff, long long vsk, VT* out2) {
    count_launch();
    launch_pdl(trace_to_kernel<T, VT>, dim3(small_grid(total)), dim3(256), st, a, b, sign, out, total, dj, joff,
               vsk, out2);
}
template <typename VT, typename T>
void launch_trace_from(const VT* in, T* out, T* out2, long long total, cudaStream_t st, const int* dj, int joff,
                       long long vsk) {
    count_launch();
    trace_from_kernel<VT, T><<<small_grid(total), 256, 0, st>>>(in, out, out2, total, dj, joff, vsk);
}
template <typename VT>
void launch_sub(const VT* b, const VT* w, VT* r, long long total, cudaStream_t st) {
    count_launch();
    sub_kernel<VT><<<small_grid(total), 256, 0, st>>>(b, w, r, total);
}
#define HELM_TRACE_INST(T, VT)                                                                                 \
    template void launch_trace_to<T, VT>(const T*, const T*, int, VT*, long long, cudaStream_t, const int*, int,  \
                                         long long, VT*);                                                      \
    template void launch_trace_from<VT, T>(const VT*, T*, T*, long long, cudaStream_t, const int*, int, long long);
HELM_TRACE_INST(float2, float2)
HELM_TRACE_INST(float2, double2)
HELM_TRACE_INST(double2, double2)
#undef HELM_TRACE_INST
template void launch_sub<float2>(const float2*, const float2*, float2*, long long, cudaStream_t);
template void launch_sub<double2>(const double2*, const double2*, double2*, long long, cudaStream_t);

// ------------------------------------------------ device-side Arnoldi loop control
// After Arnoldi step ctl[0] = j of a device-driven FGMRES cycle: every active RHS
// counts the step (iters, jcount = j + 1) and stops at est <= thr (tol ||b||), at
// ctl[2] (maxit) steps or on a non-finite estimate; the loop goes on while some RHS
// is active, j + 1 < ctl[1] (the restart length) and no device wait expired.
__global__ void arnoldi_ctl_kernel(int* ctl, const double* est, const double* thr, int* active, int* iters,
                                   int* jcount, int nrhs, const int* err, cudaGraphConditionalHandle h) {
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    const int j = ctl[0], maxit = ctl[2];
    for (int k = threadIdx.x; k < nrhs; k += blockDim.x) {
        if (!active[k]) continue;
        const int it = iters[k] + 1;
        iters[k] = it;
        jcount[k] = j + 1;
        const double e = est[k];
        if (e <= thr[k] || it >= maxit || !isfinite(e)) active[k] = 0;
        else atomicOr(&any, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int jn = j + 1;
        ctl[0] = jn;
        const bool more = any && jn < ctl[1] && *err == 0;
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}
void launch_arnoldi_ctl(int* ctl, const double* est, const double* thr, int* active, int* iters, int* jcount,
                        int maxit, int nrhs, const int* err, cudaGraphConditionalHandle h, cudaStream_t st) {
    count_launch();
    (void)maxit;   // read on the device from ctl[2]: one graph serves every maxit
    launch_pdl(arnoldi_ctl_kernel, dim3(1), dim3(256), st, ctl, est, thr, active, iters, jcount, nrhs, err, h);
}
