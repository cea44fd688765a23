// Batched block-tridiagonal factorisation of the subdomain matrices.
//
// The local matrix of Eq. subPbm on an mx x my node box, ordered row by row,
// is block tridiagonal: tridiag(-I, D_r, -I) with D_r = tridiag(-1, d_r, -1)
// (d_r: the local diagonal including the ghost coefficients of the outer and
// interface sides).  Its block LU with identity upper-diagonal blocks is
//
//     T_1 = D_1,   X_r = T_r^{-1},   T_{r+1} = D_{r+1} - X_r,
//
// so a solve needs only the X_r (the row-by-row Schur complements).  Every
// T_r is complex symmetric, hence so is X_r; the stored X_r is symmetrised.
// One CTA per subdomain runs the m_y sequential inversions; each inversion
// is an in-place Gauss-Jordan elimination with partial (row) pivoting,
// undone by column interchanges at the end.
#include "helm_internal.cuh"

namespace {

constexpr int FT = 1024;   // threads per CTA

template <typename T> __device__ __forceinline__ T cinv(T a) {
    auto d = a.x * a.x + a.y * a.y;
    return mk(a.x / d, -a.y / d);
}

template <typename R>
__global__ void __launch_bounds__(FT) factor_kernel(const SubDev* __restrict__ subtab, const double2* __restrict__ dloc,
                                                    Cx<R>* __restrict__ X, Cx<R>* __restrict__ work,
                                                    size_t work_stride, int use_smem, int* __restrict__ info) {
    using T = Cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SubDev sd = subtab[blockIdx.x];
    const int m = sd.mx, my = sd.my;
    const int w0 = sd.w0, ld0 = sd.ld0, ld1 = sd.ld1;
    const long long xr_elems = (long long)m * (ld0 + ld1);
    // element (i, j) of a stored X_r (two column halves)
    auto xidx = [&](int i, int j) -> long long {
        return j < w0 ? (long long)i * ld0 + j : (long long)m * ld0 + (long long)i * ld1 + (j - w0);
    };
    const int tid = threadIdx.x;
    T* W = use_smem ? reinterpret_cast<T*>(smem_raw) : work + blockIdx.x * work_stride;
    unsigned char* tail = smem_raw + (use_smem ? (size_t)m * m * sizeof(T) : 0);
    T* colk = reinterpret_cast<T*>(tail);                       // m entries
    int* piv = reinterpret_cast<int*>(tail + (size_t)m * sizeof(T));   // m entries
    __shared__ int s_p;
    __shared__ T s_inv;
    int fail = 0;

    for (int r = 0; r < my; ++r) {
        // T_r = D_r - X_{r-1}
        const double2* d = dloc + sd.loff + (long long)r * m;
        const T* Xp = X + sd.xoff + (long long)(r - 1) * xr_elems;
        for (int idx = tid; idx < m * m; idx += FT) {
            const int i = idx / m, j = idx - i * m;
            T v = czero<T>();
            if (r > 0) {
                const T xp = Xp[xidx(i, j)];
                v = mk(-xp.x, -xp.y);
            }
            if (i == j) v = cadd(v, from_c128<T>(d[i]));
            else if (i - j == 1 || j - i == 1) v.x -= (R)1;
            W[idx] = v;
        }
        __syncthreads();

        // in-place Gauss-Jordan with partial pivoting
        for (int k = 0; k < m; ++k) {
            if (tid < 32) {
                R best = (R)-1;
                int bi = k;
                for (int i = k + tid; i < m; i += 32) {
                    R a = cabs2(W[(long long)i * m + k]);
                    if (a > best) { best = a; bi = i; }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    R ob = __shfl_down_sync(0xffffffffu, best, o);
                    int oi = __shfl_down_sync(0xffffffffu, bi, o);
                    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
                }
                if (tid == 0) {
                    s_p = bi;
                    piv[k] = bi;
                    if (best <= (R)0 && !fail) fail = r * m + k + 1;
                }
            }
            __syncthreads();
            const int p = s_p;
            if (p != k) {
                for (int j = tid; j < m; j += FT) {
                    T t = W[(long long)k * m + j];
                    W[(long long)k * m + j] = W[(long long)p * m + j];
                    W[(long long)p * m + j] = t;
                }
            }
            __syncthreads();
            if (tid == 0) {
                T pv = W[(long long)k * m + k];
                s_inv = cabs2(pv) > (R)0 ? cinv(pv) : czero<T>();
            }
            for (int i = tid; i < m; i += FT) colk[i] = W[(long long)i * m + k];
            __syncthreads();
            const T inv = s_inv;
            for (int j = tid; j < m; j += FT)
                W[(long long)k * m + j] = (j == k) ? inv : cmul(W[(long long)k * m + j], inv);
            __syncthreads();
            for (int idx = tid; idx < m * m; idx += FT) {
                const int i = idx / m, j = idx - i * m;
                if (i == k) continue;
                const T f = colk[i];
                if (j == k) W[idx] = mk(-(f.x * inv.x - f.y * inv.y), -(f.x * inv.y + f.y * inv.x));
                else W[idx] = cfma(mk(-f.x, -f.y), W[(long long)k * m + j], W[idx]);
            }
            __syncthreads();
        }
        // undo the row interchanges: swap columns in reverse order
        for (int k = m - 1; k >= 0; --k) {
            const int p = piv[k];
            if (p != k) {
                for (int i = tid; i < m; i += FT) {
                    T t = W[(long long)i * m + k];
                    W[(long long)i * m + k] = W[(long long)i * m + p];
                    W[(long long)i * m + p] = t;
                }
            }
            __syncthreads();
        }
        // X_r = (W + W^T)/2 in the two-half layout, padding columns zeroed
        T* Xr = X + sd.xoff + (long long)r * xr_elems;
        for (long long idx = tid; idx < xr_elems; idx += FT) {
            int i, j;
            bool pad;
            if (idx < (long long)m * ld0) {
                i = (int)(idx / ld0);
                const int jj = (int)(idx - (long long)i * ld0);
                j = jj;
                pad = jj >= w0;
            } else {
                const long long t2 = idx - (long long)m * ld0;
                i = (int)(t2 / ld1);
                const int jj = (int)(t2 - (long long)i * ld1);
                j = w0 + jj;
                pad = j >= m;
            }
            T v = czero<T>();
            if (!pad) v = cscale(cadd(W[(long long)i * m + j], W[(long long)j * m + i]), (R)0.5);
            Xr[idx] = v;
        }
        __syncthreads();
    }
    if (tid == 0) info[blockIdx.x] = fail;
}

}  // namespace

template <typename R>
cudaError_t launch_factor(const SubDev* subtab, int nsub, int max_mx, const double2* dloc, Cx<R>* X,
                          Cx<R>* work, size_t work_stride, int* info, cudaStream_t st) {
    using T = Cx<R>;
    const size_t mat = (size_t)max_mx * max_mx * sizeof(T);
    const size_t tail = (size_t)max_mx * (sizeof(T) + sizeof(int));
    const size_t limit = 227 * 1024 - 1024;
    const int use_smem = (mat + tail <= limit) ? 1 : 0;
    const size_t smem = (use_smem ? mat : 0) + tail;
    if (!use_smem && work == nullptr) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(factor_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launch();
    factor_kernel<R><<<nsub, FT, smem, st>>>(subtab, dloc, X, work, work_stride, use_smem, info);
    return cudaGetLastError();
}

// factor workspace needed in global memory (0 when the matrix fits in shared memory)
size_t factor_work_elems(int max_mx, size_t elem) {
    const size_t mat = (size_t)max_mx * max_mx * elem;
    const size_t tail = (size_t)max_mx * (elem + sizeof(int));
    return (mat + tail <= 227 * 1024 - 1024) ? 0 : (size_t)max_mx * max_mx;
}

template cudaError_t launch_factor<float>(const SubDev*, int, int, const double2*, float2*, float2*, size_t, int*,
                                          cudaStream_t);
template cudaError_t launch_factor<double>(const SubDev*, int, int, const double2*, double2*, double2*, size_t,
                                           int*, cudaStream_t);
