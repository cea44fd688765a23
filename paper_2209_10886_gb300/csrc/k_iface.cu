// Interface stages of the sweep schedule: every stage whose local problems
// have zero volume source and whose only output is the outgoing interface
// data (the sweep steps of Sections 4-5 and the residual half-step of the
// block Jacobi update).  For such a stage the local solve followed by the
// trace restriction is the linear map
//
//     u_b = K (cin o G_in),        K = (A_loc^{-1}) restricted to the interface
//                                      boundary points (rows and columns),
//
// and the outgoing data is G_out = ca G_in + cb u_b (the scaled form of
// (-d_{n_{i,j}} - T) u_i, Eq. subPbm), i.e. one application of the paper's
// local scattering operators S_{m(j,i),m(i,k)} of subdomain i (Section 3).
// K is built once per factorisation by batched multi-RHS block solves
// (k_stage.cu, basis mode).  This kernel gathers the incoming traces, runs the
// GEMV with a warp per output row, applies the transmission and scatters the
// results into the neighbours' slots.
#include "helm_internal.cuh"

namespace {

constexpr int IT = 256;      // threads per CTA
constexpr int RB = 16;       // output rows per CTA

template <typename R, int NR>
__global__ void __launch_bounds__(IT) iface_kernel(IfaceArgs<R> a) {
    using T = Cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const SubDev sd = a.subtab[a.subs[blockIdx.x]];
    const int Lb = sd.Lb;
    const int rhs0 = blockIdx.z * NR;
    const int nr = min(NR, a.nrhs - rhs0);
    const int len[4] = {sd.my, sd.my, sd.mx, sd.mx};
    // output rows: points of the masked interface sides, in the order W, E, S, N
    int rcount = 0;
    for (int s = 0; s < 4; ++s)
        if ((a.mask & (1 << s)) && sd.bo[s] >= 0) rcount += len[s];
    const int row0 = blockIdx.y * RB;
    if (row0 >= rcount) return;

    T* graw = reinterpret_cast<T*>(smem_raw);      // [NR][Lb] incoming data
    T* g = graw + (size_t)NR * Lb;                 // [NR][Lb] cin * incoming data
    for (int idx = threadIdx.x; idx < NR * Lb; idx += IT) {
        const int k = idx / Lb, e = idx - k * Lb;
        int s = 0;
        while (s < 3 && !(sd.bo[s] >= 0 && e >= sd.bo[s] && e < sd.bo[s] + len[s])) ++s;
        const long long ti = sd.tin[s] + (e - sd.bo[s]);
        T G = czero<T>(), Gs = czero<T>();
        if (k < nr) {
            const long long o = (long long)(rhs0 + k) * a.ntrace + ti;
            if (a.gin0) G = a.gin0[o];
            if (a.gin1) G = cadd(G, a.gin1[o]);
            Gs = cmul(G, a.tc[ti].cin);
        }
        graw[idx] = G;
        g[idx] = Gs;
    }
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const T* K = a.K + sd.koff;
    for (int rr = warp; rr < RB; rr += IT / 32) {
        const int row = row0 + rr;
        if (row >= rcount) break;
        int s = 0, pt = row;
        for (; s < 4; ++s) {
            if (!((a.mask & (1 << s)) && sd.bo[s] >= 0)) continue;
            if (pt < len[s]) break;
            pt -= len[s];
        }
        const int krow = sd.bo[s] + pt;
        const T* Kr = K + (long long)krow * Lb;
        T acc[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[k] = czero<T>();
#pragma unroll 4
        for (int c = lane; c < Lb; c += 32) {
            const T kv = Kr[c];
#pragma unroll
            for (int k = 0; k < NR; ++k) acc[k] = cfma(kv, g[k * Lb + c], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < NR; ++k)
            for (int o = 16; o > 0; o >>= 1) {
                acc[k].x += __shfl_down_sync(0xffffffffu, acc[k].x, o);
                acc[k].y += __shfl_down_sync(0xffffffffu, acc[k].y, o);
            }
        if (lane == 0) {
            const long long ti = sd.tin[s] + pt, to = sd.tout[s] + pt;
            const TraceCoef<T> c = a.tc[ti];
            for (int k = 0; k < nr; ++k) {
                T out = cfma(c.cb, acc[k], cmul(c.ca, graw[k * Lb + krow]));
                const long long o = (long long)(rhs0 + k) * a.ntrace + to;
                if (a.base) out = cadd(out, a.base[o]);
                if (a.sub) out = csub(out, a.sub[o]);
                a.dst[o] = out;
                if (a.dst2) a.dst2[o] = out;
            }
        }
    }
}

template <typename R, int NR>
cudaError_t launch_nr(const IfaceArgs<R>& a, int nactive, int max_rows, int max_Lb, cudaStream_t st) {
    using T = Cx<R>;
    const size_t smem = 2 * (size_t)NR * max_Lb * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(iface_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(nactive, (max_rows + RB - 1) / RB, (a.nrhs + NR - 1) / NR);
    count_launch();
    iface_kernel<R, NR><<<grid, IT, smem, st>>>(a);
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_iface(const IfaceArgs<R>& a, int nactive, int max_rows, int max_Lb, cudaStream_t st) {
    if (nactive == 0 || a.nrhs == 0) return cudaSuccess;
    // blocks of 4 RHS: wider blocks (8, 16) re-read K less often but leave fewer CTAs
    // and measured slower (16 RHS: 2x the time at 64 RHS on the 1023^2 workload)
    if (a.nrhs >= 4) return launch_nr<R, 4>(a, nactive, max_rows, max_Lb, st);
    if (a.nrhs >= 2) return launch_nr<R, 2>(a, nactive, max_rows, max_Lb, st);
    return launch_nr<R, 1>(a, nactive, max_rows, max_Lb, st);
}

template cudaError_t launch_iface<float>(const IfaceArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_iface<double>(const IfaceArgs<double>&, int, int, int, cudaStream_t);
