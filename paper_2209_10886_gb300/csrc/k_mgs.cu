// Modified Gram-Schmidt step of the FP64 Arnoldi process in one persistent,
// cooperatively launched kernel.
//
// For every right-hand side: w <- w - sum_k h_k v_k with h_k = v_k^H w taken
// against the current w (modified Gram-Schmidt: 4 FP64 FMA per element for the
// dot and 4 for the update of each basis vector, half of classical
// Gram-Schmidt with reorthogonalisation), then h_{j+1,j} = ||w|| and
// v_{j+1} = w / ||w||.  Each CTA keeps its slice of w in registers for the
// whole process; each projection reads its slice of v_k once from HBM (the
// update re-reads it from L1).  The dot products are reduced deterministically:
// every CTA writes its partial sum, passes a grid barrier, and adds all
// partials in the same order.  Barrier waits are bounded in time; on expiry the
// kernel records HELM_ERR_TIMEOUT and returns.
#include "helm_internal.cuh"

namespace {

constexpr int MT = 256;                          // threads per CTA
constexpr long long BAR_LIMIT = 2000000000LL;    // cycles (~1 s)

struct MgsArgs {
    const double2* V;          // basis: v_k of RHS r at V + k*vsk + r*vsr
    long long vsk, vsr;
    double2* w;                // new vector of RHS r at w + r*vsr (overwritten by v_{j+1})
    int nvec;                  // j + 1 basis vectors to project out
    long long n;
    int nrhs;
    const int* active;
    double2* hcol;             // h_k of RHS r at hcol[r*ldh + k]
    int ldh;
    double* hnorm;             // ||w|| after the projections, per RHS
    double2* partial;          // [2 * gridDim.x] scratch of partial sums
    unsigned* bar;             // [0] arrival count, [1] generation (zero before the first launch)
    int* err;
};

__device__ __forceinline__ double2 warp_sum2(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// grid-wide barrier over co-resident CTAs; returns false when the wait expired
__device__ bool grid_barrier(unsigned* bar, int* err, int* sflag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > BAR_LIMIT) {
                    atomicExch(err, (int)HELM_ERR_TIMEOUT);
                    *sflag = 1;
                    break;
                }
            }
        }
        __threadfence();
    }
    __syncthreads();
    return *sflag == 0;
}

// sum of the gridDim.x partials in a fixed order, broadcast to the CTA
__device__ double2 sum_partials(const double2* partial, double2* sh) {
    double2 t = make_double2(0.0, 0.0);
    if (threadIdx.x < 32) {
        for (int c = threadIdx.x; c < (int)gridDim.x; c += 32) {
            const double2 v = __ldcg(partial + c);
            t.x += v.x;
            t.y += v.y;
        }
        t = warp_sum2(t);
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

// block sum of a complex value into partial[blockIdx.x]
__device__ void block_partial(double2 v, double2* partial, double2* sh) {
    v = warp_sum2(v);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[1 + wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int i = 0; i < MT / 32; ++i) { t.x += sh[1 + i].x; t.y += sh[1 + i].y; }
        partial[blockIdx.x] = t;
    }
}

template <int EPT>
__global__ void __launch_bounds__(MT) mgs_kernel(MgsArgs a) {
    __shared__ double2 sh[1 + MT / 32];
    __shared__ int sflag;
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * MT;
    const long long base = (long long)blockIdx.x * MT + threadIdx.x;
    // reduction s writes partial[(s & 1) * gridDim.x + cta]: a CTA can only write
    // reduction s+1 after every CTA has passed barrier s, i.e. has read reduction
    // s-1 (which used the other half), so one barrier per reduction suffices
    unsigned s = 0;
    auto reduce = [&](double2 v, double2& out) -> bool {
        double2* part = a.partial + (s & 1u) * gridDim.x;
        block_partial(v, part, sh);
        if (!grid_barrier(a.bar, a.err, &sflag)) return false;
        out = sum_partials(part, sh);
        ++s;
        return true;
    };
    for (int r = 0; r < a.nrhs; ++r) {
        if (a.active && !a.active[r]) continue;
        double2* w = a.w + r * a.vsr;
        double2 wr[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const long long p = base + e * stride;
            wr[e] = p < a.n ? w[p] : make_double2(0.0, 0.0);
        }
        // step k: finish the update with v_{k-1} (h_{k-1} known) and, in the same
        // pass over the elements, the dot product with v_k against the updated w
        double2 mh = make_double2(0.0, 0.0);
        const double2* vprev = nullptr;
        for (int k = 0; k < a.nvec; ++k) {
            const double2* v = a.V + k * a.vsk + r * a.vsr;
            double2 acc = make_double2(0.0, 0.0);
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const long long p = base + e * stride;
                if (p < a.n) {
                    if (vprev) wr[e] = cfma(mh, vprev[p], wr[e]);
                    acc = cfmaconj(v[p], wr[e], acc);
                }
            }
            double2 h;
            if (!reduce(acc, h)) return;
            if (blockIdx.x == 0 && threadIdx.x == 0) a.hcol[(long long)r * a.ldh + k] = h;
            mh = make_double2(-h.x, -h.y);
            vprev = v;
        }
        double nrm = 0.0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const long long p = base + e * stride;
            if (vprev && p < a.n) wr[e] = cfma(mh, vprev[p], wr[e]);
            nrm = fma(wr[e].x, wr[e].x, fma(wr[e].y, wr[e].y, nrm));
        }
        double2 tot;
        if (!reduce(make_double2(nrm, 0.0), tot)) return;
        const double hn = sqrt(tot.x);
        if (blockIdx.x == 0 && threadIdx.x == 0) a.hnorm[r] = hn;
        const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const long long p = base + e * stride;
            if (p < a.n) w[p] = make_double2(wr[e].x * inv, wr[e].y * inv);
        }
    }
}

template <int EPT>
cudaError_t launch_ept(MgsArgs& a, int grid, cudaStream_t st) {
    void* args[] = {&a};
    count_launch();
    return cudaLaunchCooperativeKernel((const void*)mgs_kernel<EPT>, dim3(grid), dim3(MT), args, 0, st);
}

}  // namespace

// Grid size (CTAs, all co-resident) for the persistent Gram-Schmidt kernel, or 0.
int mgs_grid() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mgs_kernel<32>, MT, 0) != cudaSuccess) return 0;
    return per >= 1 ? sms : 0;
}

// largest vector length the register-resident kernel handles with `grid` CTAs
long long mgs_max_n(int grid) { return (long long)grid * MT * 32; }

// w <- (w - V V^H w) / ||.|| by modified Gram-Schmidt for every active RHS.
cudaError_t launch_mgs(const double2* V, long long vsk, long long vsr, double2* w, int nvec, long long n, int nrhs,
                       const int* active, double2* hcol, int ldh, double* hnorm, double2* partial, unsigned* bar,
                       int* err, int grid, cudaStream_t st) {
    MgsArgs a{V, vsk, vsr, w, nvec, n, nrhs, active, hcol, ldh, hnorm, partial, bar, err};
    const long long per = (n + (long long)grid * MT - 1) / ((long long)grid * MT);
    if (per <= 4) return launch_ept<4>(a, grid, st);
    if (per <= 8) return launch_ept<8>(a, grid, st);
    if (per <= 16) return launch_ept<16>(a, grid, st);
    if (per <= 32) return launch_ept<32>(a, grid, st);
    return cudaErrorInvalidValue;
}
