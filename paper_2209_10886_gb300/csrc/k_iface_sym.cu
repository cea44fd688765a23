// The stages that apply every subdomain's whole boundary operator (the block Jacobi
// residual and the interface operator S), one complex64 RHS, from packed symmetric
// boundary operators.
//
// The boundary operator of a subdomain, K = P^T A_loc^{-1} P (the local solve
// restricted to the interface boundary points, before the transmission
// coefficients of Section 3's scattering operators are applied), is complex
// symmetric because the local matrix is: the five-point rows and their Robin
// diagonal terms are symmetric.  Its upper triangle, stored as 32 x 32 tiles,
// takes half the bytes of the full operator: on the 1023^2, 8 x 8 workload 67
// instead of 134 MB, which the 129 MB L2 can hold across the interface
// iterations, while the full operator does not fit.
//
// Persistent streaming form: each CTA owns a contiguous range of output row tiles
// (subdomain, tile row I of 32 boundary points) and computes them completely, so no
// CTA waits for another.  Row tile I needs the stored tiles (I, J) for J >= I and
// (J, I) for J < I; one producer thread streams them, in J order, by bulk copies into
// shared memory, starting before the dependency wait (K does not change during a
// solve).  Consumer warp w takes the tiles J = w, w + 8, ..., through a slot of its own
// (each slot is filled and emptied in one warp's order, so a parity wait never looks
// more than one phase ahead):
// lane l accumulates output row l, from a stored (I, J) tile along its row l (read
// diagonally skewed, so that the 32 lanes hit distinct banks) and from a stored
// (J, I) tile down its column l.  The warps' sums are added in warp order and the
// outgoing data formed from per-point terms prepared with the gather:
//     G_out = cb u_b + (ca G_in + base - sub).
#include "helm_internal.cuh"

#include <algorithm>

namespace {

constexpr int TB = SYM_TB;

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

// measured on the 1023^2, 8 x 8 workload: 8 consumer warps with one slot each at two
// CTAs per SM (22.0 ms per solve); 4 warps at 3 or 4 CTAs per SM, or two slots per warp,
// within 1 %; one CTA per SM (16 slots) 24.4-24.9 ms
constexpr int CW = 8;                         // consumer warps
constexpr int D = 1;                          // tile slots (8 KB) per consumer warp
constexpr int CTAS = 2;                       // CTAs per SM
constexpr int SLOTS = CW * D;
constexpr int ST = 32 * (CW + 1);             // + one producer warp
constexpr long long SYM_WAIT = 2000000000LL;  // cycles (~1 s) before a wait gives up

__device__ __forceinline__ unsigned sm32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(unsigned long long* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sm32(b)) : "memory");
}
__device__ __forceinline__ void mb_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sm32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(sm32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait for the phase with this parity (limit 0: one look)
__device__ __forceinline__ bool mb_wait(unsigned long long* b, unsigned parity, long long limit) {
    if (mb_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mb_try(b, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void consumers_sync() { asm volatile("bar.sync 1, %0;\n" ::"r"(32 * CW) : "memory"); }

// rt[t] = (subdomain id, tile row I) of output row tile t, subdomain by subdomain;
// dynamic shared memory: slot[CW][1024] | gc[gcap] (cin * G_in) | cb[gcap] | cterm[gcap]
__global__ void __launch_bounds__(ST, CTAS) iface_sym_kernel(IfaceArgs<float> a, const int2* rt, int nrt, int gcap) {
    using T = float2;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) unsigned long long full[SLOTS], empty[SLOTS];
    __shared__ T ys[CW][TB];
    __shared__ int abort_flag;
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    T* ring = reinterpret_cast<T*>(smem);
    T* gc = ring + (size_t)SLOTS * TB * TB;
    T* cbv = gc + gcap;
    T* ctv = cbv + gcap;
    const int t0 = (int)((long long)blockIdx.x * nrt / gridDim.x);
    const int t1 = (int)((long long)(blockIdx.x + 1) * nrt / gridDim.x);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int i = 0; i < SLOTS; ++i) {
            mb_init(&full[i]);
            mb_init(&empty[i]);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    if (t0 >= t1) return;

    if (warp == CW) {
        // producer: the tiles of every row tile of the range, in order
        if (lane != 0) return;
        int fills[CW];                    // tiles sent through each warp's slot so far
#pragma unroll
        for (int v = 0; v < CW; ++v) fills[v] = 0;
        for (int t = t0; t < t1 && !*((volatile int*)&abort_flag); ++t) {
            const int2 w = HLD(rt + t);
            const SubDev sd = HLD(a.subtab + w.x);
            const int nt = (sd.Lb + TB - 1) / TB, I = w.y;
            const T* Kb = a.Kp + sd.kpoff;
            for (int J = 0; J < nt; ++J) {
                const int cw = J % CW;
                int n = 0;
#pragma unroll
                for (int v = 0; v < CW; ++v)
                    if (v == cw) n = fills[v];
                const int slot = cw * D + n % D;
                // the warp has emptied the slot's previous tile (its fill n / D - 1)
                if (n >= D && !mb_wait(&empty[slot], (unsigned)((n / D - 1) & 1), SYM_WAIT)) {
                    abort_flag = 1;
                    if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
                    break;
                }
#pragma unroll
                for (int v = 0; v < CW; ++v)
                    if (v == cw) fills[v] = n + 1;
                const T* src = Kb + (J >= I ? tile_off(nt, I, J) : tile_off(nt, J, I));
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sm32(&full[slot])),
                             "r"(TB * TB * 8)
                             : "memory");
                if (HELM_CHK(src, TB * TB * sizeof(T)))   // checking build: the wait then gives up
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                            sm32(ring + (size_t)slot * TB * TB)),
                        "l"(src), "r"(TB * TB * 8), "r"(sm32(&full[slot]))
                        : "memory");
            }
        }
        // no copy outlives the CTA: on abort, wait (bounded) for the last fill of each slot
        if (*((volatile int*)&abort_flag))
#pragma unroll
            for (int v = 0; v < CW; ++v)
                for (int q = fills[v] - 1; q >= 0 && q >= fills[v] - D; --q)
                    mb_wait(&full[v * D + q % D], (unsigned)((q / D) & 1), SYM_WAIT);
        return;
    }

    // consumers
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    int n = 0, cur = -1;                  // tiles this warp has taken from its slot
    for (int t = t0; t < t1; ++t) {
        const int2 w = HLD(rt + t);
        const SubDev sd = HLD(a.subtab + w.x);
        const int Lb = sd.Lb, nt = (Lb + TB - 1) / TB, I = w.y;
        const int bo[4] = {sd.bo[0], sd.bo[1], sd.bo[2], sd.bo[3]};
        const int tin[4] = {sd.tin[0], sd.tin[1], sd.tin[2], sd.tin[3]};
        const int tout[4] = {sd.tout[0], sd.tout[1], sd.tout[2], sd.tout[3]};
        if (w.x != cur) {
            // a new subdomain: cin * G_in, cb and the constant term of every boundary point
            for (int e = threadIdx.x; e < nt * TB; e += 32 * CW) {
                T g = czero<T>(), cb = czero<T>(), ct = czero<T>();
                if (e < Lb) {
                    const int s = side_of(bo, e);
                    const int pt = e - pick4(bo, s);
                    const long long ti = pick4(tin, s) + pt, to = pick4(tout, s) + pt;
                    const TraceCoef<T> c = HLD(a.tc + ti);
                    T G = czero<T>();
                    if (a.gin0) G = HLD(a.gin0 + ti);
                    if (a.gin1) G = cadd(G, HLD(a.gin1 + ti));
                    T bsub = czero<T>();
                    if (a.base) bsub = HLD(a.base + to);
                    if (a.sub) bsub = csub(bsub, HLD(a.sub + to));
                    g = cmul(G, c.cin);
                    cb = c.cb;
                    ct = cadd(cmul(c.ca, G), bsub);
                }
                gc[e] = g;
                cbv[e] = cb;
                ctv[e] = ct;
            }
            consumers_sync();
            cur = w.x;
        }
        T acc = czero<T>();
        for (int J = warp; J < nt; J += CW, ++n) {
            const int slot = warp * D + n % D;
            const bool ab = *((volatile int*)&abort_flag) != 0;
            if (!mb_wait(&full[slot], (unsigned)((n / D) & 1), ab ? 0 : SYM_WAIT)) {
                abort_flag = 1;
                if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
            }
            if (!*((volatile int*)&abort_flag)) {
                const T* tile = ring + (size_t)slot * TB * TB;
                const T* gJ = gc + J * TB;
                if (J >= I) {
                    // stored (I, J): row `lane` of the tile, diagonally
#pragma unroll 8
                    for (int cc = 0; cc < TB; ++cc) {
                        const int c = (cc + lane) & (TB - 1);
                        acc = cfma(tile[lane * TB + c], gJ[c], acc);
                    }
                } else {
                    // stored (J, I): column `lane` of the tile
#pragma unroll 8
                    for (int r = 0; r < TB; ++r) acc = cfma(tile[r * TB + lane], gJ[r], acc);
                }
            }
            __syncwarp();
            if (lane == 0) mb_arrive(&empty[slot]);
        }
        ys[warp][lane] = acc;
        consumers_sync();
        if (warp == 0 && !*((volatile int*)&abort_flag)) {
            T y = ys[0][lane];
#pragma unroll
            for (int v = 1; v < CW; ++v) y = cadd(y, ys[v][lane]);
            const int e = I * TB + lane;
            if (e < Lb) {
                const int s = side_of(bo, e);
                const long long to = pick4(tout, s) + (e - pick4(bo, s));
                const T out = cadd(cmul(cbv[e], y), ctv[e]);
                HST(a.dst + to, out);
                if (a.dst2) HST(a.dst2 + to, out);
            }
        }
        consumers_sync();                 // ys, and at a new subdomain the point terms, are reused
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

cudaError_t launch_iface_sym(const IfaceArgs<float>& a, const int2* rt, int nrt, int max_Lb, int num_sms,
                             cudaStream_t st) {
    if (nrt == 0 || a.nrhs == 0) return cudaSuccess;
    if (a.nrhs != 1 || !a.Kp || !rt || a.mask != 15 || max_Lb < 1 || max_Lb > SYM_MAXLB) return cudaErrorInvalidValue;
    const int gcap = (max_Lb + TB - 1) / TB * TB;
    const size_t smem = (size_t)SLOTS * TB * TB * sizeof(float2) + 3 * (size_t)gcap * sizeof(float2);
    cudaError_t e = cudaFuncSetAttribute(iface_sym_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::min(nrt, CTAS * std::max(1, num_sms)));
    cfg.blockDim = dim3(ST);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, iface_sym_kernel, a, rt, nrt, gcap);
}
