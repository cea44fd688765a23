// Internal declarations shared by the CUDA translation units of libhelm.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>
#include <vector>

#include "helm.h"
#include "helm_check.cuh"

// ----------------------------------------------------------------- complex
// float2 / double2 carry complex64 / complex128 values (re, im).
template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using T = float2; };
template <> struct CplxOf<double> { using T = double2; };
template <typename R> using Cx = typename CplxOf<R>::T;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
template <typename T> __host__ __device__ __forceinline__ T czero();
template <> __host__ __device__ __forceinline__ float2 czero<float2>() { return make_float2(0.f, 0.f); }
template <> __host__ __device__ __forceinline__ double2 czero<double2>() { return make_double2(0.0, 0.0); }

template <typename T> __host__ __device__ __forceinline__ T cadd(T a, T b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T> __host__ __device__ __forceinline__ T csub(T a, T b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T> __host__ __device__ __forceinline__ T cmul(T a, T b) {
    return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// acc + a*b
template <typename T> __host__ __device__ __forceinline__ T cfma(T a, T b, T acc) {
    return mk(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}
// acc + conj(a)*b
template <typename T> __host__ __device__ __forceinline__ T cfmaconj(T a, T b, T acc) {
    return mk(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
template <typename T, typename S> __host__ __device__ __forceinline__ T cscale(T a, S s) { return mk(a.x * s, a.y * s); }
template <typename T> __host__ __device__ __forceinline__ auto cabs2(T a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ float2 to_c64(double2 a) { return make_float2((float)a.x, (float)a.y); }
__device__ __forceinline__ double2 to_c128(float2 a) { return make_double2((double)a.x, (double)a.y); }
__device__ __forceinline__ double2 to_c128(double2 a) { return a; }
// Column j of the Arnoldi least-squares problem through the Givens rotations, in
// the precision of C2 (double2; float2 where the Krylov vectors are complex64 and
// the least-squares problem needs no more).  On entry col[0..j] = h_{0..j,j},
// col[j+1] = h_{j+1,j}, cs[0..j) (cosines, real parts) and sn[0..j) hold the
// earlier rotations and gj = g_j of the rotated right-hand side, all in fast
// memory: the chain of rotations is serial, so the caller converts precisions
// beforehand (conversions run on GB300's narrow FP64 pipe).  Applies rotations
// 0..j-1, forms rotation j so that it zeroes col[j+1], stores it in cs[j], sn[j]
// and returns the new g_j, g_{j+1} (|g_{j+1}| is the residual estimate).  A
// rotation acts as [a; b] <- [c a + s b; -conj(s) a + c b].
template <typename C2>
__device__ inline void givens_column(C2* col, C2* cs, C2* sn, int j, C2& gj, C2& gj1) {
    using Re = decltype(C2::x);
    Re ax = col[0].x, ay = col[0].y;                 // the running upper entry of the pair
    for (int i = 0; i < j; ++i) {
        const C2 b = col[i + 1];
        const Re c = cs[i].x;
        const C2 s = sn[i];
        col[i] = mk(c * ax + (s.x * b.x - s.y * b.y), c * ay + (s.x * b.y + s.y * b.x));
        const Re nx = c * b.x - (s.x * ax + s.y * ay);
        const Re ny = c * b.y - (s.x * ay - s.y * ax);
        ax = nx;
        ay = ny;
    }
    const C2 b = col[j + 1];
    const Re na = sqrt(ax * ax + ay * ay), nb = sqrt(b.x * b.x + b.y * b.y);
    const Re den = sqrt(na * na + nb * nb);
    Re c;
    C2 s;
    if (den == (Re)0) { c = 1; s = mk((Re)0, (Re)0); }
    else if (na == (Re)0) { c = 0; s = mk(b.x / den, -b.y / den); }          // conj(b)/|b|
    else {
        c = na / den;
        const Re px = ax / na, py = ay / na;                                    // a/|a|
        s = mk((px * b.x + py * b.y) / den, (py * b.x - px * b.y) / den);       // ph*conj(b)/den
    }
    cs[j] = mk(c, (Re)0);
    sn[j] = s;
    col[j] = mk(c * ax + (s.x * b.x - s.y * b.y), c * ay + (s.x * b.y + s.y * b.x));
    col[j + 1] = mk((Re)0, (Re)0);
    const C2 g0 = gj;
    gj1 = mk(-(s.x * g0.x + s.y * g0.y), -(s.x * g0.y - s.y * g0.x));          // -conj(s) g_j
    gj = mk(c * g0.x, c * g0.y);
}
template <typename T> __device__ __forceinline__ T from_c128(double2 a);
template <> __device__ __forceinline__ float2 from_c128<float2>(double2 a) { return to_c64(a); }
template <> __device__ __forceinline__ double2 from_c128<double2>(double2 a) { return a; }

// complex division a/b in double (setup-time only)
__host__ __device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// ------------------------------------------------------------------ tables
enum Side { SW = 0, SE = 1, SS = 2, SN = 3 };   // neighbour direction: west, east, south, north

// One subdomain as the kernels see it.
struct SubDev {
    int x0, y0, mx, my;        // node box origin and size (0-based global nodes)
    // each stored X_r is two column halves, each row-major: columns [0, w0) with
    // leading dimension ld0, then columns [w0, mx) with leading dimension ld1
    // (element (i, j) at i*ld0 + j, or mx*ld0 + i*ld1 + (j - w0))
    int w0, ld0, ld1;
    int tin[4];                // start of the incoming slot (this, neighbour) in the trace buffer, -1: outer side
    int tout[4];               // start of the slot (neighbour, this) that receives this subdomain's outgoing data
    long long xoff;            // element offset of X_1 of this subdomain in the factor array
    long long yoff;            // element offset of this subdomain's block in the solve workspace (per RHS)
    long long loff;            // offset of the node block in the local-diagonal array
    // interface boundary vector of this subdomain: the points of its interface
    // sides in the order W, E, S, N (outer sides skipped); bo[s] = offset of
    // side s in it (-1: outer side), Lb = its length
    int bo[4];
    int Lb;
    long long koff;            // element offset of the Lb x Lb boundary operator K in its array
    long long kpoff;           // element offset of K's packed symmetric tiles (k_iface_sym.cu)
    long long xtoff;           // float offset of this subdomain's factors in the tensor-core layout (k_tc.cu)
    int tcmt;                  // 128-node tiles of that layout: 1 (mx <= 128), 2 (mx <= 256), 0 (wider)
    long long eoff;            // offset of this subdomain's 2 (mx + my) boundary slots in the edge scratch
};

// Trace-point coefficients of one interface edge point (beta_e = T_e h / 2):
//   cin = 1/(1-beta)                (incoming data -> local right-hand side)
//   ca  = -(1+beta)/(1-beta)        (outgoing data: G_out = ca*G_in + cb*u_p)
//   cb  = -4 beta/(1-beta)
template <typename T> struct TraceCoef { T cin, ca, cb; };

// Interface-buffer identifiers used by the stage lists.
// BUF_U (HABC transmission only): the boundary values of the liftings' base solves,
// kept from the lifting to the reconstruction
enum Buf { BUF_NONE = -1, BUF_B = 0, BUF_X = 1, BUF_Y = 2, BUF_U = 3 };

struct StageDesc {
    int iface;                 // 1: zero volume source and no volume output: boundary-operator GEMV
    std::vector<int> subs;     // subdomains solved in this stage
    int src;                   // 1: volume source r_i, 0: zero source
    int in0, in1;              // incoming data = in0 (+ in1), Buf ids
    int mask;                  // bit s set: emit outgoing data toward side s
    int dst, dst2, base, sub;  // dst[slot] = base[slot] - sub[slot] + G_out (also into dst2)
    int final_;                // 1: write the volume solution into z
    int sub_off;               // offset of `subs` in the device stage-list array
    int tc_off[2], tc_n[2];    // the same subdomains split by tensor-core tile count (1, 2): offsets, counts
    int kmat = 0;              // interface stages: the per-subdomain matrix they apply (KMAT_*)
};
// matrices of the interface stages: K (or, with the HABC transmission, Q), and the
// HABC lifting (Lq) and reconstruction (D1 on the incoming data, D2 on the lifting's
// boundary values) maps
enum { KMAT_K = 0, KMAT_LQ = 1, KMAT_D1 = 2, KMAT_D2 = 3 };

// launch parameters of the fused stage kernel (passed by value)
template <typename R> struct StageArgs {
    using T = Cx<R>;
    const SubDev* subtab;
    const int* subs;           // active subdomain ids for this stage
    int nx, ny;                // global grid
    int nrhs;                  // right-hand sides in the batch
    long long ntrace;          // trace points per RHS
    long long wstride;         // solve-workspace elements per RHS
    const T* X;                // factors
    const TraceCoef<T>* tc;    // per trace point
    int src;
    const double2* r;          // source fields (c128), RHS stride nx*ny
    const double* rscale;      // per-RHS factor applied to r (1/||r|| for c64), or null = 1
    const T* gin0; const T* gin1;
    int mask;
    T* dst; T* dst2; const T* base; const T* sub;
    double2* z;                // volume output (final stage) or null
    const double* zscale;      // per-RHS factor applied to the output, or null = 1
    T* yws;                    // solve workspace
    // basis mode (boundary operator construction): RHS k of CTA column block y is
    // the unit datum at interface boundary point col0 + y*NR + k; the boundary
    // values of the solution are stored as that row of K
    T* K;
    int col0;
    int* err;                  // device status word: set to HELM_ERR_TIMEOUT when a bounded wait expires
    // tensor-core path: per RHS, estride boundary slots (W[my] E[my] S[mx] N[mx] of every
    // subdomain at SubDev::eoff): escr = interface data of the nodes, uscr = boundary values
    T* escr;
    T* uscr;
    long long estride;
    const T* r64;              // tensor-core path: the source already scaled by rscale, in complex64
};

// launch parameters of the interface (boundary-operator) stage kernel
template <typename R> struct IfaceArgs {
    using T = Cx<R>;
    const SubDev* subtab;
    const int* subs;
    int nrhs;
    long long ntrace;
    const T* K;
    const TraceCoef<T>* tc;
    const T* gin0; const T* gin1;
    int mask;
    T* dst; T* dst2; const T* base; const T* sub;
    void* bufs[3];             // sweep kernel: the interface buffers B, X, Y the stages name
    int* err;                  // HELM_ERR_TIMEOUT when a bounded wait expired
    // tensor-core form split over the boundary points: partial accumulators (part_cap
    // floats) and one arrival counter per output tile (cnt_cap, zero between launches)
    float* part; long long part_cap;
    int* cnt; int cnt_cap;
    // packed symmetric form (complex64, one RHS, k_iface_sym.cu): the upper-triangle tiles
    // of every K
    const T* Kp;
};

// output rows of one work item of an interface stage (host tables and kernels agree on it)
constexpr int IFACE_RB = 16;

// launch shape of the interface-stage kernel: right-hand sides per block (1, 2, 4, 8, 16),
// K rows staged in shared memory when they fit (1) or read from global memory (0), and
// the CTAs per SM the grid aims at when it spreads RHS blocks over CTAs
struct IfaceCfg {
    int nr = 4, staged = 1, waves = 3;
    // complex64 only: tc = 3 or 1 runs the stages of at least tc_min_ctas CTAs (-1: two per
    // SM) as tensor-core MMAs (3xTF32 or TF32 operands, tc_iface_kernel) with tc_nb = 16 or
    // 32 RHS per CTA, the smaller stages with the CUDA-core shape above; tc = 0: CUDA cores
    int tc = 0, tc_nb = 16, tc_min_ctas = -1;
};

// one interface stage of a sweep run by the persistent sweep kernel (device table)
struct SweepStage {
    int sub_off, nsub;         // its subdomains in the stage-list array
    int in0, in1, mask, dst, dst2, base, sub;   // Buf ids (-1: none), as in StageDesc
    int max_rows;              // the most output rows (masked-side points) of one of its subdomains
};

// ------------------------------------------------------------ launch count
void count_launch(int n = 1);

// ------------------------------------------------------------ error helpers
void set_error(const std::string& msg);
helm_status cuda_status(cudaError_t e, const char* what);

#define HELM_CUDA_TRY(expr)                                            \
    do {                                                               \
        cudaError_t _e = (expr);                                       \
        if (_e != cudaSuccess) return cuda_status(_e, #expr);          \
    } while (0)

// --------------------------------------------------------------- launchers
// setup kernels
void launch_setup_coeffs(const double* m2, int nx, int ny, double h, double omega,
                         const int* xcut, const int* ycut, int N1, int N2, const int* subid,
                         int transmission, double tc_scale,
                         double2* adiag, double2* dloc, const SubDev* subtab, cudaStream_t st);
void launch_trace_coeffs(const double* m2, int nx, double h, double omega, int transmission,
                         double tc_scale, const int* slot_sub, const int* slot_side, const int* slot_off,
                         const int* slot_len, int nslots, const SubDev* subtab,
                         TraceCoef<double2>* tc128, TraceCoef<float2>* tc64, cudaStream_t st);
// factor
template <typename R>
cudaError_t launch_factor(const SubDev* subtab, int nsub, int max_mx, const double2* dloc,
                          Cx<R>* X, Cx<R>* work, size_t work_stride, int* info, cudaStream_t st);
// stage
// max_w: widest column half, max_ld: largest half leading dimension, num_sms: SMs of the device
// launch shape of the full-stage kernels chosen by the autotuner (0: the kernel's rule):
// csize CTAs per subdomain (1, 2), factor chunk of chunk_kb KB per ring slot (64, 48,
// 32), tensor-core form tc_nr RHS per CTA (16, 32, 64)
struct StageCfg { int csize = 0, chunk_kb = 0, tc_nr = 0; };
template <typename R>
cudaError_t launch_stage(const StageArgs<R>& a, int nactive, int max_mx, int max_my, int max_w, int max_ld,
                         int num_sms, cudaStream_t st, const StageCfg* cfg = nullptr);
// boundary operators K of all subdomains, columns [col0, col0 + ncols) per launch
template <typename R>
cudaError_t launch_basis(const StageArgs<R>& a, int nsub, int ncols, int max_mx, int max_my, int max_w, int max_ld,
                         cudaStream_t st);
// tensor-core (TF32) multi-RHS solves of complex64 factors (k_tc.cu)
// split = 3: operands as hi + lo TF32 pairs, three MMAs per product; split = 1: TF32 alone.
// Every subdomain has its own tile count (SubDev::tcmt); one launch covers the
// subdomains a.subs[0 .. nactive) of tile count MT.
int tc_tiles(int mx);                                     // 128-node M tiles (1 or 2), 0: unsupported width
long long tc_layout_floats(int mx, int my, int MT, int split);   // floats of one subdomain's factors in that layout
cudaError_t launch_tc_layout(const SubDev* subtab, int nsub, int split, const float2* X, float* XT, cudaStream_t st);
// complex64 factorisation with the Gauss-Jordan trailing updates on the tensor cores
// (3xTF32); every subdomain at most 128 nodes wide
cudaError_t launch_tc_factor(const SubDev* subtab, int nsub, const double2* dloc, float2* X, int* info, int* err,
                             cudaStream_t st);
cudaError_t launch_tc_stage(const StageArgs<float>& a, const float* XT, int MT, int split, int nactive,
                            cudaStream_t st, int nr = 0);   // nr: RHS per CTA (0: the rule)
cudaError_t launch_iface_tc(const IfaceArgs<float>& a, int nactive, int max_rows, int split, int nb, int min_ctas,
                            int max_Lb, cudaStream_t st);
cudaError_t launch_tc_basis(const StageArgs<float>& a, const float* XT, int MT, int split, int nsub, int ncols,
                            cudaStream_t st);
// one interface stage; cfg = nullptr: the default shape (4, 2 or 1 RHS per block, staged
// when it fits, 3 CTAs per SM)
template <typename R>
cudaError_t launch_iface(const IfaceArgs<R>& a, int nactive, int max_rows, int max_Lb, cudaStream_t st,
                         const IfaceCfg* cfg = nullptr);
// the interface stages of a sweep as one dependency-driven cooperative launch: items
// (stage, subdomain index in the stage, row block, counter id) in stage order; counter u
// completes after need[u] items; unit_deps[u] = (offset, count) of its list in deps;
// counters zero on entry
template <typename R>
cudaError_t launch_sweep_dep(const IfaceArgs<R>& a, const SweepStage* stages, const int4* items, int nitems,
                             const int* need, const int2* unit_deps, const int* deps, int* counters, int max_Lb,
                             cudaStream_t st);
// Packed symmetric boundary operators (k_iface_sym.cu).  K = P^T A_loc^{-1} P is complex
// symmetric (A_loc is); its upper triangle is stored in SYM_TB x SYM_TB tiles, tile row
// by tile row, tile (I, J >= I) at kpoff + (I nt - I (I - 1) / 2 + J - I) SYM_TB^2, zero
// past Lb (nt = ceil(Lb / SYM_TB) <= 32)
constexpr int SYM_TB = 32;
constexpr int SYM_MAXLB = 1024;
__host__ __device__ __forceinline__ long long sym_tiles(int Lb) {
    const long long nt = (Lb + SYM_TB - 1) / SYM_TB;
    return nt * (nt + 1) / 2;
}
// Kp = the symmetric part (K + K^T) / 2 of every subdomain's K, packed as above
cudaError_t launch_sym_pack(const SubDev* subtab, int nsub, int ntmax, const float2* K, float2* Kp, cudaStream_t st);
// one complex64 interface stage with one RHS over every subdomain and all four sides
// (a.mask = 15) from the packed operators (a.Kp set); rt: the nrt output row tiles
// (subdomain id, tile row), subdomain by subdomain; the same outputs as launch_iface up to
// rounding
cudaError_t launch_iface_sym(const IfaceArgs<float>& a, const int2* rt, int nrt, int max_Lb, int num_sms,
                             cudaStream_t st);
// a whole sweep (nstages interface stages, in order) in one cooperative launch of `grid`
// CTAs (sweep_grid: the co-resident count, 0 when unavailable); bar: two zeroed words
template <typename R> int sweep_grid(int nrhs, int max_Lb);
template <typename R>
cudaError_t launch_sweep(const IfaceArgs<R>& a, const SweepStage* stages, int nstages, int max_Lb, int grid,
                         unsigned* bar, int* err, cudaStream_t st);
// krylov / vector kernels
void launch_matvec(const double2* adiag, int nx, int ny, const double2* u, double2* Au, int nrhs,
                   cudaStream_t st);
int launch_residual(const double2* adiag, int nx, int ny, const double2* f, double fscale,
                     const double2* u, double2* r, int nrhs, const int* active, double* partial,
                     int nblk, cudaStream_t st);
// VT: double2 or float2 (partial sums and coefficients FP64 in both)
template <typename VT>
void launch_norm2_partial(const VT* v, long long n, int nrhs, long long stride, double* partial,
                          int nblk, cudaStream_t st);
void launch_reduce_rows(const double* partial, int nblk, int nrows, double* out, int mode,
                        cudaStream_t st);
template <typename VT>
void launch_mdot(const VT* V, long long vstride_k, long long vstride_rhs, int nvec,
                 const VT* w, long long wstride, long long n, int nrhs, const int* active,
                 double2* partial, int nblk, cudaStream_t st);
void launch_reduce_cpartials(const double2* partial, int nblk, int nrows, double2* out,
                             long long out_stride, int nrhs, cudaStream_t st);
template <typename VT>
void launch_mupdate(const VT* V, long long vstride_k, long long vstride_rhs, int nvec,
                    const int* nvec_rhs, const double2* coef, long long coef_stride, double sign, VT* w,
                    long long wstride, long long n, int nrhs, const int* active, double* norm_partial,
                    int nblk, cudaStream_t st);
template <typename VT>
void launch_scale_vec(VT* dst, long long dstride, const VT* src, long long sstride,
                      const double* inv, long long n, int nrhs, const int* active, cudaStream_t st);
void launch_hessenberg_step(double2* H, int ldh, long long hstride, double2* cs, double2* sn, double2* g,
                            int ldg, const double2* hcol, long long hcol_stride, const double* hnorm,
                            int j, int nrhs, const int* active, double* resid_est, double* inv_hnext,
                            cudaStream_t st);
void launch_hessenberg_solve(const double2* H, int ldh, long long hstride, const double2* g, int ldg,
                             const int* jcount, double2* y, int ldy, int nrhs, cudaStream_t st);
void launch_mask_copy(double2* dst, const double2* src, long long n, int nrhs, const int* active,
                      cudaStream_t st);
void launch_sqrt_inplace(double* v, int n, cudaStream_t st);
// interface vectors (T = the trace buffers' complex type, VT = the Krylov vectors'):
// out = sign (a + b) (b optional, sign +1 or -1); out (and out2) = in rounded to T; r = b - w
template <typename T, typename VT>
void launch_trace_to(const T* a, const T* b, int sign, VT* out, long long total, cudaStream_t st,
                     const int* dj = nullptr, int joff = 0, long long vsk = 0, VT* out2 = nullptr);
template <typename VT, typename T>
void launch_trace_from(const VT* in, T* out, T* out2, long long total, cudaStream_t st, const int* dj = nullptr,
                       int joff = 0, long long vsk = 0);
template <typename VT>
void launch_sub(const VT* b, const VT* w, VT* r, long long total, cudaStream_t st);
// out[k*n + i] = complex64(src[k*n + i] * scale[k])
void launch_to_c64_scaled(const double2* src, const double* scale, float2* out, long long n, int nrhs,
                          cudaStream_t st);
void launch_scale_from_norm(const double* norm2, double* inv, double* scale, int n, cudaStream_t st);
// device-driven Arnoldi loop: step bookkeeping and the loop condition (ctl[0] = j, ctl[1] = restart)
void launch_arnoldi_ctl(int* ctl, const double* est, const double* thr, int* active, int* iters, int* jcount,
                        int maxit, int nrhs, const int* err, cudaGraphConditionalHandle h, cudaStream_t st);
// HABC transmission (k_habc.cu): side operators M_s = I - (h/2) T_s per slot, batched
// Gauss-Jordan inversion, batched complex GEMM, the precomputed stage matrices, and the
// trace swap (slot (i, j) <-> (j, i))
cudaError_t launch_habc_sides(const double* m2, int nx, double h, double omega, int n_pade, double phi,
                              const int* slot_sub, const int* slot_side, const int* slot_len,
                              const long long* slot_moff, int nslots, int max_len, const SubDev* subtab, double2* M,
                              double2* Y, cudaStream_t st);
int gj_grid(int maxn);
size_t gj_mat_bytes();
void gj_mat_fill(void* dst, int i, double2* A, int n, int lda);
cudaError_t launch_gj_inverse(const void* mats, int nmat, int maxn, double2* pub, unsigned* bar, int* err, int* info,
                              cudaStream_t st);
size_t gemm_prob_bytes();
void gemm_prob_fill(void* dst, int i, const double2* A, const double2* B, double2* C, int m, int n, int k, int lda,
                    int ldb, int ldc, double2 alpha, int accumulate);
cudaError_t launch_zgemm_batched(const void* probs, int nprob, int max_m, int max_n, cudaStream_t st);
size_t habc_sub_bytes();
void habc_sub_fill(void* dst, int i, long long koff, long long toff, int Lb, const int* bo, const int* len,
                   const long long* moff, const int* tin);
template <typename T>
cudaError_t launch_habc_form(const void* subs, int nsub, int max_Lb, const T* K, const TraceCoef<double2>* tc,
                             double2* K64, const double2* KR, double2* W, int phase, cudaStream_t st);
template <typename T>
cudaError_t launch_habc_final(const void* subs, int nsub, int max_Lb, const double2* Mside,
                              const TraceCoef<double2>* tc, const double2* P1, const double2* RP, const double2* W,
                              const double2* RW, T* Q, T* Lq, T* D1, T* D2, cudaStream_t st);
template <typename T>
void launch_trace_swap(const T* in, T* out, const int* swp, long long ntrace, int nrhs, cudaStream_t st);
// adjoint
void launch_receiver_residual(const double2* u, long long N, const int* rec, int nrec, const double2* d,
                              int nsrc, double2* res, double* partial, cudaStream_t st);
void launch_adjoint_rhs(const double2* res, const int* rec, int nrec, int nsrc, long long N,
                        double inv_h2, double2* f_adj, cudaStream_t st);
void launch_gradient(const double2* U, const double2* Lt, const double* m2, int nx, int ny, double h,
                     double omega, int nsrc, double* grad, cudaStream_t st);
