// Interface stages from the packed symmetric boundary operators (complex64, one RHS).
//
// The boundary operator of a subdomain, K = P^T A_loc^{-1} P (the local solve
// restricted to the interface boundary points, before the transmission
// coefficients of Section 3's scattering operators are applied), is complex
// symmetric because the local matrix is: the five-point rows and their Robin
// diagonal terms are symmetric.  Its upper triangle, stored as 32 x 32 tiles,
// takes half the bytes of the full operator: on the 1023^2, 8 x 8 workload 67
// instead of 134 MB, which stays resident in the 129 MB L2 across the interface
// iterations, while the full operator does not fit and streams from HBM at
// every stage that applies all of it.
//
// One CTA per (subdomain, row tile I) reads each stored tile (I, J >= I) that
// the stage needs once and uses it twice: K_IJ g_J adds to the outputs of row
// tile I (a per-lane partial over the tile's columns, summed over the warp by a
// butterfly reduce-scatter) and, for J > I, K_IJ^T g_I adds to those of row tile
// J (one output per lane, no reduction).  The contributions to row tile J come
// from the CTAs I <= J; each writes its partial vector into its own slot and
// counts its arrival, and the CTA that arrives last for J adds the J + 1
// partials in the order of I and forms the outgoing data
//     G_out = ca G_in + cb u_b + (base - sub)
// for the points of J that lie on masked sides.  No CTA waits for another, and
// the sums do not depend on the order of arrival.
#include "helm_internal.cuh"

namespace {

constexpr int TB = SYM_TB;
constexpr int NW = 8;              // warps per CTA
constexpr int NT = 32 * NW;

__device__ __forceinline__ int pick4(const int (&v)[4], int s) {
    return s == 0 ? v[0] : s == 1 ? v[1] : s == 2 ? v[2] : v[3];
}
// side of interface boundary point e: the last interface side starting at or before it
__device__ __forceinline__ int side_of(const int (&bo)[4], int e) {
    int s = 0;
#pragma unroll
    for (int q = 1; q < 4; ++q)
        if (bo[q] >= 0 && e >= bo[q]) s = q;
    return s;
}
// element offset of stored tile (I, J), J >= I, of a subdomain with nt row tiles
__host__ __device__ __forceinline__ long long tile_off(int nt, int I, int J) {
    return ((long long)I * nt - (long long)I * (I - 1) / 2 + (J - I)) * (TB * TB);
}

__global__ void __launch_bounds__(256) sym_pack_kernel(const SubDev* subtab, const float2* K, float2* Kp) {
    const SubDev sd = HLD(subtab + blockIdx.x);
    const int Lb = sd.Lb, nt = (Lb + TB - 1) / TB;
    const int I = blockIdx.y, J = blockIdx.z;
    if (I >= nt || J >= nt || J < I) return;
    float2* dst = Kp + sd.kpoff + tile_off(nt, I, J);
    const float2* Ks = K + sd.koff;
    for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
        const int i = I * TB + idx / TB, j = J * TB + idx % TB;
        float2 v = make_float2(0.f, 0.f);
        if (i < Lb && j < Lb) {
            const float2 x = HLD(Ks + (long long)i * Lb + j), y = HLD(Ks + (long long)j * Lb + i);
            v = make_float2(0.5f * (x.x + y.x), 0.5f * (x.y + y.y));
        }
        HST(dst + idx, v);
    }
}

__global__ void __launch_bounds__(NT, 2) iface_sym_kernel(IfaceArgs<float> a) {
    using T = float2;
    __shared__ T gs[SYM_MAXLB];        // cin * incoming data of every boundary point, zero past Lb
    __shared__ T ys[NW][TB];           // the warps' partial outputs of row tile I
    __shared__ int jobs[32];           // row tiles this CTA completes
    __shared__ int njobs;
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int sid = HLD(a.subs + blockIdx.x);
    const SubDev sd = HLD(a.subtab + sid);
    const int Lb = sd.Lb, nt = (Lb + TB - 1) / TB;
    const int I = blockIdx.y;
    if (I >= nt) return;
    const int bo[4] = {sd.bo[0], sd.bo[1], sd.bo[2], sd.bo[3]};
    const int tin[4] = {sd.tin[0], sd.tin[1], sd.tin[2], sd.tin[3]};
    const int tout[4] = {sd.tout[0], sd.tout[1], sd.tout[2], sd.tout[3]};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // row tiles holding points of masked sides
    unsigned M = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (((a.mask >> s) & 1) && bo[s] >= 0) {
            const int len = s < 2 ? sd.my : sd.mx;
            for (int t = bo[s] / TB; t <= (bo[s] + len - 1) / TB; ++t) M |= 1u << t;
        }
    const bool rowI = (M >> I) & 1u;
    // the stored tiles (I, J) this CTA applies: all of tile row I when I is masked, else
    // the ones whose transposed product feeds a masked row tile
    unsigned need = 0;
    for (int J = I; J < nt; ++J)
        if (rowI || ((M >> J) & 1u)) need |= 1u << J;
    if (need == 0) return;
    const int ntile = __popc(need);
    auto nth = [&](int k) {            // the k-th set bit of need
        unsigned m = need;
        for (int q = 0; q < k; ++q) m &= m - 1;
        return __ffs(m) - 1;
    };
    const T* Kb = a.Kp + sd.kpoff;
    // K does not change during the solve: start the first tile of each warp on its way
    // into L1 while the previous stage may still run
    if (warp < ntile) {
        const char* t0 = reinterpret_cast<const char*>(Kb + tile_off(nt, I, nth(warp))) + lane * 256;
        asm volatile("prefetch.global.L1 [%0];\n" ::"l"(t0));
        asm volatile("prefetch.global.L1 [%0];\n" ::"l"(t0 + 128));
    }
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    // cin * (G_in0 + G_in1) of every boundary point
    for (int e = threadIdx.x; e < nt * TB; e += NT) {
        T g = czero<T>();
        if (e < Lb) {
            const int s = side_of(bo, e);
            const long long ti = pick4(tin, s) + (e - pick4(bo, s));
            T G = czero<T>();
            if (a.gin0) G = HLD(a.gin0 + ti);
            if (a.gin1) G = cadd(G, HLD(a.gin1 + ti));
            g = cmul(G, HLD(a.tc + ti).cin);
        }
        gs[e] = g;
    }
    __syncthreads();

    const long long slot0 = (long long)sid * a.ntmax;          // this subdomain's row tiles
    T p[TB];                                                    // direct partials of row tile I
#pragma unroll
    for (int r = 0; r < TB; ++r) p[r] = czero<T>();
    const T* gI = gs + I * TB;
    for (int k = warp; k < ntile; k += NW) {
        const int J = nth(k);
        const T* tile = Kb + tile_off(nt, I, J) + lane;
        const bool trn = J > I && ((M >> J) & 1u);
        const T gJ = gs[J * TB + lane];
        T q = czero<T>();
#pragma unroll
        for (int r0 = 0; r0 < TB; r0 += 16) {
            T kv[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const T* kp = tile + (r0 + u) * TB;
                kv[u] = HELM_CHK(kp, sizeof(T)) ? __ldg(kp) : czero<T>();
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                if (rowI) p[r0 + u] = cfma(kv[u], gJ, p[r0 + u]);
                if (trn) q = cfma(kv[u], gI[r0 + u], q);
            }
        }
        if (trn) HST(a.spart + ((slot0 + J) * a.ntmax + I) * TB + lane, q);
    }
    if (rowI) {
        // reduce-scatter over the lanes: lane l ends with the warp's sum of p[l]
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const bool up = (lane & o) != 0;
#pragma unroll
            for (int i = 0; i < o; ++i) {
                const T send = up ? p[i] : p[i + o];
                const T keep = up ? p[i + o] : p[i];
                p[i] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, o),
                                   keep.y + __shfl_xor_sync(0xffffffffu, send.y, o));
            }
        }
        ys[warp][lane] = p[0];
    }
    __syncthreads();
    if (rowI && warp == 0) {
        T y = ys[0][lane];
#pragma unroll
        for (int w = 1; w < NW; ++w) y = cadd(y, ys[w][lane]);
        HST(a.spart + ((slot0 + I) * a.ntmax + I) * TB + lane, y);
    }
    // count this CTA's contributions (row tiles J >= I that are masked); the CTA that
    // brings the (J + 1)-th one completes row tile J
    __threadfence();
    if (threadIdx.x == 0) njobs = 0;
    __syncthreads();
    if (threadIdx.x < nt) {
        const int J = threadIdx.x;
        if (J >= I && ((M >> J) & 1u)) {
            const int old = HELM_CHK(a.scnt + slot0 + J, sizeof(int)) ? atomicAdd(a.scnt + slot0 + J, 1) : -1;
            if (old == J) jobs[atomicAdd(&njobs, 1)] = J;
        }
    }
    __syncthreads();
    const int nj = njobs;
    if (nj == 0) return;
    __threadfence();
    for (int jb = warp; jb < nj; jb += NW) {
        const int J = jobs[jb];
        const T* pj = a.spart + (slot0 + J) * a.ntmax * TB + lane;
        T y = czero<T>();
        for (int i = 0; i <= J; ++i) {
            const T* pi = pj + (long long)i * TB;
            y = cadd(y, HELM_CHK(pi, sizeof(T)) ? __ldcg(pi) : czero<T>());
        }
        const int e = J * TB + lane;
        if (e < Lb) {
            const int s = side_of(bo, e);
            if ((a.mask >> s) & 1) {
                const int pt = e - pick4(bo, s);
                const long long ti = pick4(tin, s) + pt, to = pick4(tout, s) + pt;
                const TraceCoef<T> c = HLD(a.tc + ti);
                T G = czero<T>();
                if (a.gin0) G = HLD(a.gin0 + ti);
                if (a.gin1) G = cadd(G, HLD(a.gin1 + ti));
                T bsub = czero<T>();
                if (a.base) bsub = HLD(a.base + to);
                if (a.sub) bsub = csub(bsub, HLD(a.sub + to));
                const T out = cadd(cfma(c.cb, y, cmul(c.ca, G)), bsub);
                HST(a.dst + to, out);
                if (a.dst2) HST(a.dst2 + to, out);
            }
        }
        if (lane == 0) HST(a.scnt + slot0 + J, 0);              // ready for the next stage
    }
}

}  // namespace

cudaError_t launch_sym_pack(const SubDev* subtab, int nsub, int ntmax, const float2* K, float2* Kp, cudaStream_t st) {
    if (nsub == 0) return cudaSuccess;
    if (ntmax < 1 || ntmax > SYM_MAXLB / SYM_TB) return cudaErrorInvalidValue;
    count_launch();
    sym_pack_kernel<<<dim3(nsub, ntmax, ntmax), 256, 0, st>>>(subtab, K, Kp);
    return cudaGetLastError();
}

cudaError_t launch_iface_sym(const IfaceArgs<float>& a, int nactive, cudaStream_t st) {
    if (nactive == 0 || a.nrhs == 0) return cudaSuccess;
    if (a.nrhs != 1 || !a.Kp || !a.spart || !a.scnt || a.ntmax < 1 || a.ntmax > SYM_MAXLB / SYM_TB)
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nactive, a.ntmax);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, iface_sym_kernel, a);
}
