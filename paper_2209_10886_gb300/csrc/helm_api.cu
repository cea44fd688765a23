// C ABI of libhelm: problem setup (partition, the paper's interface
// numbering, coefficient tables), the sweep schedules as lists of batched
// stages, the preconditioner driver, FP64 flexible GMRES and the adjoint
// misfit gradient.  See include/helm.h for the contract of each entry point.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "helm_internal.cuh"

// NVTX ranges around the entry points and every stage (header-only NVTX v3: each call
// is a no-op unless a profiler injects its library)
#if __has_include(<nvtx3/nvToolsExt.h>)
#include <nvtx3/nvToolsExt.h>
#define HELM_HAVE_NVTX 1
#endif
namespace {
struct NvtxRange {
    explicit NvtxRange(const char* name) {
#ifdef HELM_HAVE_NVTX
        nvtxRangePushA(name);
#else
        (void)name;
#endif
    }
    ~NvtxRange() {
#ifdef HELM_HAVE_NVTX
        nvtxRangePop();
#endif
    }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
}  // namespace

// ------------------------------------------------------------ bounds-checking build
// The live device ranges the kernels may touch: every allocation of the library (the
// cudaMalloc / cudaFree calls of this file go through hc_malloc / hc_free) and the
// caller's buffers of the call in progress (HcCall).  Every change is uploaded to the
// range table of each translation unit before the next launch.
#ifdef HELM_CHECK_BOUNDS
#include <mutex>
namespace {
struct HcUnit {
    HcUpload up;
    HcRead rd;
    HcReset rs;
    const char* file;
};
struct HcState {
    std::mutex mu;
    std::vector<HcUnit> units;
    std::map<unsigned long long, unsigned long long> allocs;        // start -> end
    std::vector<std::pair<unsigned long long, unsigned long long>> call;
};
HcState& hc() {
    static HcState s;
    return s;
}
cudaError_t hc_upload_locked(HcState& s) {
    static HcTable t;
    t.n = 0;
    auto add = [&](unsigned long long lo, unsigned long long hi) {
        if (lo < hi && t.n < HC_MAX_RANGES) t.r[t.n++] = {lo, hi};
    };
    for (auto& a : s.allocs) add(a.first, a.second);
    for (auto& c : s.call) add(c.first, c.second);
    cudaError_t e = cudaSuccess;
    for (auto& u : s.units)
        if (e == cudaSuccess) e = u.up(t);
    return e;
}
cudaError_t hc_malloc(void** p, size_t n) {
    const cudaError_t e = cudaMalloc(p, n);
    if (e != cudaSuccess || !*p) return e;
    HcState& s = hc();
    std::lock_guard<std::mutex> g(s.mu);
    const unsigned long long lo = reinterpret_cast<unsigned long long>(*p);
    s.allocs[lo] = lo + n;
    return hc_upload_locked(s);
}
cudaError_t hc_free(void* p) {
    {
        HcState& s = hc();
        std::lock_guard<std::mutex> g(s.mu);
        s.allocs.erase(reinterpret_cast<unsigned long long>(p));
        (void)hc_upload_locked(s);
    }
    return cudaFree(p);
}
}  // namespace
void hc_register_unit(HcUpload up, HcRead rd, HcReset rs, const char* file) {
    HcState& s = hc();
    std::lock_guard<std::mutex> g(s.mu);
    s.units.push_back({up, rd, rs, file});
}
namespace {
// the caller's buffers of one entry point, for the duration of the call
struct HcCall {
    size_t keep;
    HcCall(std::initializer_list<std::pair<const void*, size_t>> bufs) {
        HcState& s = hc();
        std::lock_guard<std::mutex> g(s.mu);
        keep = s.call.size();
        for (auto& b : bufs)
            if (b.first && b.second) {
                const unsigned long long lo = reinterpret_cast<unsigned long long>(b.first);
                s.call.push_back({lo, lo + b.second});
            }
        (void)hc_upload_locked(s);
    }
    ~HcCall() {
        HcState& s = hc();
        std::lock_guard<std::mutex> g(s.mu);
        s.call.resize(keep);
    }
    HcCall(const HcCall&) = delete;
    HcCall& operator=(const HcCall&) = delete;
};
}  // namespace
#define cudaMalloc(pp, n) hc_malloc((void**)(pp), (n))
#define cudaFree(p) hc_free((void*)(p))
#else
namespace {
struct HcCall {
    HcCall(std::initializer_list<std::pair<const void*, size_t>>) {}
};
}  // namespace
#endif

extern "C" int helm_check_bounds_report(long long* violations, unsigned long long* first_addr,
                                        long long* first_bytes, int* first_line, char* unit, int unit_len,
                                        int reset) {
#ifdef HELM_CHECK_BOUNDS
    HcState& s = hc();
    std::lock_guard<std::mutex> g(s.mu);
    long long total = 0;
    bool have = false;
    for (auto& u : s.units) {
        HcBad b{};
        if (u.rd(b) != cudaSuccess) return -1;
        total += (long long)b.count;
        if (b.count && !have) {
            have = true;
            if (first_addr) *first_addr = b.addr;
            if (first_bytes) *first_bytes = (long long)b.bytes;
            if (first_line) *first_line = b.line;
            if (unit && unit_len > 0) snprintf(unit, (size_t)unit_len, "%s", u.file);
        }
        if (reset && u.rs() != cudaSuccess) return -1;
    }
    if (violations) *violations = total;
    if (!have) {
        if (first_addr) *first_addr = 0;
        if (first_bytes) *first_bytes = 0;
        if (first_line) *first_line = 0;
        if (unit && unit_len > 0) unit[0] = 0;
    }
    return 1;
#else
    (void)first_addr; (void)first_bytes; (void)first_line; (void)unit; (void)unit_len; (void)reset;
    if (violations) *violations = 0;
    return 0;
#endif
}

#ifdef HELM_CHECK_BOUNDS
namespace {
__global__ void hc_selftest_kernel(const unsigned char* buf, int* out) {
    out[0] = HELM_CHK(buf, 256);          // the whole allocation
    out[1] = HELM_CHK(buf + 256, 1);      // the byte past its end
    out[2] = HELM_CHK(buf + 255, 2);      // straddles its end
}
}  // namespace
#endif

extern "C" int helm_check_bounds_selftest(int* results) {
#ifdef HELM_CHECK_BOUNDS
    unsigned char* buf = nullptr;
    int* out = nullptr;
    if (cudaMalloc(&buf, 256) != cudaSuccess) return -1;
    if (cudaMalloc(&out, 3 * sizeof(int)) != cudaSuccess) { cudaFree(buf); return -1; }
    hc_selftest_kernel<<<1, 1>>>(buf, out);
    cudaError_t e = cudaMemcpy(results, out, 3 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(out);
    cudaFree(buf);
    return e == cudaSuccess ? 1 : -1;
#else
    (void)results;
    return 0;
#endif
}

size_t factor_work_elems(int max_mx, size_t elem);
int mgs_grid();
long long mgs_max_n(int grid);
// limit: cycles a grid barrier waits before it gives up (0: the default, ~1 s)
cudaError_t launch_mgs(const double2* V, long long vsk, long long vsr, double2* w, int nvec, long long n, int nrhs,
                       const int* active, double2* hcol, int ldh, double* hnorm, double2* partial, unsigned* bar,
                       int* err, int grid, cudaStream_t st, long long limit);
template <typename VT>
int cgs2_grid(long long n, int max_j);
template <typename VT>
cudaError_t launch_cgs2_step(const VT* V, long long vsk, long long vsr, int j, long long n, int nrhs,
                             const int* active, double2* hsum, int ldh, double* hnorm, int* need, double2* H, int ldH,
                             long long hs, double2* cs, double2* sn, double2* g, int ldg, double* est, double* invh,
                             double2* partial, unsigned* bar, int* err, int grid, cudaStream_t st,
                             const int* dj = nullptr, int jmax = 0, const VT* wsrc = nullptr,
                             VT* vout1 = nullptr, VT* vout2 = nullptr, long long limit = 0,
                             double eta2 = 0.5);

// ------------------------------------------------------------ launch count
#include <atomic>
static std::atomic<long long> g_launches{0};
void count_launch(int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
static void uncount_launch(long long n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
extern "C" long long helm_launch_count(void) { return g_launches.load(); }

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }
helm_status cuda_status(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? HELM_ERR_OOM : HELM_ERR_CUDA;
}
static helm_status arg_error(const std::string& m) {
    set_error(m);
    return HELM_ERR_ARG;
}

// ------------------------------------------------------------ schedule (S1)
namespace {

struct SubHost {
    int i1, i2;          // 1-based column, row
    int diag;            // i1 + i2
    SubDev dev;
};

// Block Jacobi bands (Section 5): forward 2+(g-1)N1 <= d <= 2+g N1, backward
// (1+Ng)-g N1 <= d <= (1+Ng)-(g-1)N1, clipped to [2, Ng+1] (consecutive bands share a
// diagonal).  overlap = false: bands of N1 diagonals that share none (the paper's
// bounds read as half-open), for comparison.
std::vector<std::pair<int, int>> bands(int N1, int Ng, bool forward, bool overlap = true) {
    std::vector<std::pair<int, int>> out;
    const int width = overlap ? N1 : N1 - 1;     // band g starts N1 diagonals after band g-1
    for (int g = 1;; ++g) {
        int lo, hi;
        if (forward) { lo = 2 + (g - 1) * N1; hi = lo + width; }
        else { hi = (1 + Ng) - (g - 1) * N1; lo = hi - width; }
        lo = std::max(lo, 2);
        hi = std::min(hi, Ng + 1);
        if (lo > Ng + 1 || hi < 2) break;
        out.push_back({lo, hi});
        if ((forward && hi >= Ng + 1) || (!forward && lo <= 2)) break;
    }
    return out;
}
static bool is_bsp(int sched) { return sched == HELM_SCHED_BSP || sched == HELM_SCHED_BSP_NONOVERLAP; }

// Stage lists of one application of the volume preconditioner.  `ondiag[d]`
// lists the subdomains of diagonal d; `all` every subdomain.
std::vector<StageDesc> build_schedule(int sched, int N1, int N2, const std::vector<std::vector<int>>& ondiag,
                                      const std::vector<int>& all, bool have_interfaces) {
    std::vector<StageDesc> st;
    const int Ng = N1 + N2 - 1;
    const int ALL = 15, FWD = (1 << SE) | (1 << SN), BWD = (1 << SW) | (1 << SS);
    auto mk_stage = [](std::vector<int> subs, int src, int in0, int in1, int mask, int dst, int dst2, int base,
                       int sub, int fin) {
        StageDesc s;
        s.iface = (src == 0 && !fin) ? 1 : 0;     // zero source, traces only: boundary-operator GEMV
        s.subs = std::move(subs);
        s.src = src; s.in0 = in0; s.in1 = in1; s.mask = mask;
        s.dst = dst; s.dst2 = dst2; s.base = base; s.sub = sub; s.final_ = fin; s.sub_off = 0;
        return s;
    };
    if (!have_interfaces) {       // one subdomain: M^{-1} = A^{-1}, one solve
        st.push_back(mk_stage(all, 1, BUF_NONE, BUF_NONE, 0, BUF_NONE, BUF_NONE, BUF_NONE, BUF_NONE, 1));
        return st;
    }
    // liftings w_i (Eq. subPbmLifting): b = outgoing of w, copied into X
    st.push_back(mk_stage(all, 1, BUF_NONE, BUF_NONE, ALL, BUF_B, BUF_X, BUF_NONE, BUF_NONE, 0));
    if (sched == HELM_SCHED_SP) {
        // S_L^{-1} = (I + E_{Ng+1}) ... (I + E_3): step d solves diagonal d-1 into d
        for (int d = 3; d <= Ng + 1; ++d)
            st.push_back(mk_stage(ondiag[d - 1], 0, BUF_X, BUF_NONE, FWD, BUF_X, BUF_NONE, BUF_B, BUF_NONE, 0));
        // S_U^{-1} = (I + F_3) ... (I + F_{Ng+1}): step d solves diagonal d into d-1
        for (int d = Ng + 1; d >= 3; --d)
            st.push_back(mk_stage(ondiag[d], 0, BUF_X, BUF_NONE, BWD, BUF_X, BUF_NONE, BUF_X, BUF_NONE, 0));
        st.push_back(mk_stage(all, 1, BUF_X, BUF_NONE, 0, BUF_NONE, BUF_NONE, BUF_NONE, BUF_NONE, 1));
        return st;
    }
    // BSP: x' = B_L^{-1} b (bands run concurrently; a band's first diagonal
    // reads the unpropagated b, later ones the propagated x)
    const bool overlap = sched != HELM_SCHED_BSP_NONOVERLAP;
    auto fb = bands(N1, Ng, true, overlap);
    int fsteps = 0;
    for (auto& b : fb) fsteps = std::max(fsteps, b.second - b.first);
    for (int s = 1; s <= fsteps; ++s) {
        std::vector<int> subs;
        for (auto& b : fb) {
            const int d = b.first + s - 1;
            if (d <= b.second - 1) subs.insert(subs.end(), ondiag[d].begin(), ondiag[d].end());
        }
        st.push_back(mk_stage(subs, 0, s == 1 ? BUF_B : BUF_X, BUF_NONE, FWD, BUF_X, BUF_NONE, BUF_B, BUF_NONE, 0));
    }
    // rho = b - (I - S) x': every subdomain, into B (in place) and Y
    st.push_back(mk_stage(all, 0, BUF_X, BUF_NONE, ALL, BUF_B, BUF_Y, BUF_B, BUF_X, 0));
    // y = B_U^{-1} rho
    auto ub = bands(N1, Ng, false, overlap);
    int bsteps = 0;
    for (auto& b : ub) bsteps = std::max(bsteps, b.second - b.first);
    for (int s = 1; s <= bsteps; ++s) {
        std::vector<int> subs;
        for (auto& b : ub) {
            const int d = b.second - s + 1;
            if (d >= b.first + 1) subs.insert(subs.end(), ondiag[d].begin(), ondiag[d].end());
        }
        st.push_back(mk_stage(subs, 0, s == 1 ? BUF_B : BUF_Y, BUF_NONE, BWD, BUF_Y, BUF_NONE, BUF_B, BUF_NONE, 0));
    }
    // reconstruction with incoming x = x' + y
    st.push_back(mk_stage(all, 1, BUF_X, BUF_Y, 0, BUF_NONE, BUF_NONE, BUF_NONE, BUF_NONE, 1));
    return st;
}

int sweep_steps(int sched, int N1, int N2) {
    const int Ng = N1 + N2 - 1;
    if (sched == HELM_SCHED_SP) return 2 * (Ng - 1);
    const bool overlap = sched != HELM_SCHED_BSP_NONOVERLAP;
    int f = 0, b = 0;
    for (auto& x : bands(N1, Ng, true, overlap)) f = std::max(f, x.second - x.first);
    for (auto& x : bands(N1, Ng, false, overlap)) b = std::max(b, x.second - x.first);
    return f + b;
}

template <typename P> cudaError_t dalloc(P*& p, size_t count) {
    p = nullptr;
    if (count == 0) return cudaSuccess;
    return cudaMalloc((void**)&p, count * sizeof(P));
}
template <typename P> void dfree(P*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

}  // namespace

// ------------------------------------------------------------------ handle
// workspace of one restarted FGMRES (V: restart+1 basis vectors, Z: restart
// preconditioned vectors, per RHS n values each; the rest per RHS and cycle)
struct KrylovWS {
    int nrhs = 0, restart = 0;
    long long n = 0;
    double2 *V = nullptr, *Z = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr;
    double2 *h1 = nullptr, *h2 = nullptr, *hsum = nullptr, *y = nullptr, *cpart = nullptr;
    double *rpart = nullptr, *rn = nullptr, *est = nullptr, *invh = nullptr;
    int *active = nullptr, *jcount = nullptr, *need = nullptr;
    double2* mgs_part = nullptr;     // partial sums of the persistent Gram-Schmidt kernel
    unsigned* mgs_bar = nullptr;     // its grid-barrier state
    double2 *b = nullptr, *x = nullptr;   // interface solver: right-hand side and solution (nrhs x n)
    int nblk = 0;
    // device-driven Arnoldi loop: ctl = {j, restart, maxit}, per-RHS step counts and stopping thresholds
    int *ctl = nullptr, *iters = nullptr;
    double* thr = nullptr;
    long long gen = 0;               // allocation generation (keys the graphs that hold these pointers)
};

struct helm_problem {
    int nx = 0, ny = 0, N1 = 0, N2 = 0;
    double h = 0, omega = 0;
    helm_setup_opts sopts{};
    std::vector<int> xcut, ycut;
    std::vector<SubHost> subs;
    std::vector<std::vector<int>> ondiag;
    std::vector<int> all;
    int max_mx = 0, max_my = 0, max_Lb = 0;
    int max_w = 0, max_ld = 0;       // widest column half and largest half leading dimension of the factors
    int num_sms = 0;
    long long ntrace = 0;
    int nslots = 0;
    std::vector<StageDesc> sched[HELM_NSCHED];

    // HABC transmission (setup option): the local problems are factored with the optimized
    // Robin condition and the HABC side blocks enter through the boundary space (k_habc.cu)
    int habc = 0;
    double2* d_rin = nullptr;        // per interface slot: Rin = (I - h T / 2)^{-1}, L x L row-major, FP64
    std::vector<long long> slot_moff;   // offset of each slot's matrix in d_rin
    std::vector<int> slot_len;
    std::map<long long, int> slot_of_toff;   // trace offset of a slot's first point -> the slot
    int* d_swap = nullptr;           // trace point -> the same point of the neighbour's slot
    TraceCoef<double2>* d_tcid128 = nullptr;   // stage coefficients with the HABC: cin = 1, ca = 0, cb = 1
    TraceCoef<float2>* d_tcid64 = nullptr;
    void* d_Lq = nullptr;            // lifting map, reconstruction maps (factor precision, K layout)
    void* d_D1 = nullptr;
    void* d_D2 = nullptr;

    double* d_m2 = nullptr;
    double2* d_adiag = nullptr;
    double2* d_dloc = nullptr;
    SubDev* d_subtab = nullptr;
    TraceCoef<double2>* d_tc128 = nullptr;
    TraceCoef<float2>* d_tc64 = nullptr;
    int* d_stage_subs = nullptr;
    int* d_err = nullptr;            // device status word written by kernels whose bounded waits expired

    int factored = 0;
    int prec = HELM_PREC_C128;
    bool tc_factor_used = false;     // the last factorisation ran its trailing updates on the tensor cores
    void* d_X = nullptr;
    void* d_K = nullptr;             // boundary operators of all subdomains
    size_t K_bytes = 0;
    // packed symmetric boundary operators (complex64, k_iface_sym.cu): the tiles, the list
    // of output row tiles (subdomain id, tile row) of all subdomains, tiles per row of the
    // largest K
    float2* d_Kp = nullptr;
    int2* d_symrt = nullptr;
    int sym_nrt = 0;
    long long kp_elems = 0;
    int sym_ntmax = 0;
    size_t X_bytes = 0;
    float* d_XT = nullptr;           // complex64 factors in the tensor cores' operand layout (k_tc.cu)
    float* d_tcpart = nullptr;       // partial sums of the tensor-core interface stages split over CTAs
    long long tcpart_cap = 0;        // floats
    int* d_tccnt = nullptr;          // their arrival counters (zero between launches)
    int tccnt_cap = 0;
    size_t XT_bytes = 0;
    int tc_mt = 0;                   // largest tile count (128 nodes each) of that layout
    int tc_split = 0;                // 3: hi + lo TF32 pairs, 1: TF32 alone
    int tc_all_off[2] = {0, 0}, tc_all_n[2] = {0, 0};   // all subdomains by tile count, in d_stage_subs
    long long etot = 0;              // boundary slots 2 (mx + my) summed over the subdomains
    SweepStage* d_sweep = nullptr;   // interface stages of each schedule for the sweep kernel
    // dependency-driven sweep: work items, per-(stage, subdomain) counters (items needed,
    // dependency list), per schedule offsets into the global arrays
    int4* d_dep_items = nullptr;
    int* d_dep_need = nullptr;
    int2* d_dep_unit = nullptr;
    int* d_dep_list = nullptr;
    int* d_dep_cnt = nullptr;
    int dep_item_off[HELM_NSCHED] = {}, dep_nitems[HELM_NSCHED] = {};
    int dep_unit_off[HELM_NSCHED] = {}, dep_nunits[HELM_NSCHED] = {};
    int sweep_off[HELM_NSCHED] = {}, sweep_n[HELM_NSCHED] = {};
    unsigned* d_sweep_bar = nullptr; // its grid-barrier words

    // preconditioner workspace
    int ws_nrhs = 0;
    void* d_trace[4] = {nullptr, nullptr, nullptr, nullptr};   // B, X, Y (and U with the HABC transmission)
    void* d_yws = nullptr;
    void* d_escr = nullptr;          // tensor-core path: 2 nrhs etot complex64 (interface data, boundary values)
    void* d_r64 = nullptr;           // tensor-core path: the scaled source in complex64 (nrhs N)
    double* d_pc_norm = nullptr;     // per RHS: ||r||^2, 1/||r||, ||r||
    double* d_pc_partial = nullptr;

    // Krylov workspaces: the volume FGMRES and the interface FGMRES nested in the preconditioner
    KrylovWS kw, kwi;
    long long inner_steps = 0;       // interface Krylov steps taken inside the preconditioner (all calls)
    int persistent = 0;              // gmres_solve option: sweeps in the persistent sweep kernel
    long long wait_cycles = 0;       // gmres_solve option: grid-barrier limit of the Gram-Schmidt kernels (0: default)
    bool inner_hist_taken = false;   // the interface history of this gmres_solve call is recorded
    struct TunedShape { int prec, nrhs; IfaceCfg cfg; };
    std::vector<TunedShape> iface_tuned;   // autotuned interface-stage launch shapes
    struct TunedStage { int prec, nrhs; StageCfg cfg; };
    std::vector<TunedStage> stage_tuned;   // autotuned full-stage launch shapes
    const StageCfg* stage_try = nullptr;   // the candidate being timed by the autotuner

    // adjoint workspace
    double2 *d_res = nullptr, *d_fadj = nullptr, *d_U = nullptr, *d_L = nullptr;
    double* d_jpart = nullptr;
    int aw_nsrc = 0, aw_nrec = 0;

    // per-kernel-class event timing (helm_profile)
    struct KProf {
        std::vector<cudaEvent_t> a, b;
        size_t used = 0;             // event pairs recorded
        long long kernels = 0;       // kernel launches inside them
        double bytes = 0;
        double flops = 0;
    };
    KProf prof[5];
    int prof_on = 0;
    // while a launch sequence is captured into a graph: its accounting per class
    int prof_capture = 0;
    double cap_bytes[5] = {0, 0, 0, 0, 0}, cap_flops[5] = {0, 0, 0, 0, 0};
    long long cap_kernels[5] = {0, 0, 0, 0, 0};

    // preconditioner applications captured as CUDA graphs (gmres_solve with use_graph):
    // one executable graph per (schedule, nrhs, r, z), replayed on the caller's stream
    struct PcGraph {
        int sched, nrhs;
        const void* r;
        void* z;
        cudaGraphExec_t exec;
        long long kernels;           // kernel launches one replay performs
        int cls = -1;                // kernel class of the sequence (profiling), -1: none
        long long cls_kernels = 0;   // its launches, algorithmic bytes and flops per replay
        double cls_bytes = 0, cls_flops = 0;
        cudaGraph_t tmpl = nullptr;  // device-loop graphs keep their template (conditional node)
        long long gen = 0;           // Krylov workspace generation a device-loop graph was built for
        int m = 0;                   // its restart length
        long long limit = 0;         // the grid-barrier limit its Gram-Schmidt launch was captured with
    };
    bool dev_loop_broken = false;    // a device-loop graph failed to build: host-driven loop from then on
    std::vector<PcGraph> graphs;
    cudaStream_t cap_stream = nullptr;
    cudaEvent_t cap_ev = nullptr;

    long long N() const { return (long long)nx * ny; }
};

// trace coefficients of the stages: the Robin ones, or with the HABC transmission the
// identity ones (cin = 1, ca = 0, cb = 1: the stage matrices carry the transmission)
template <typename T> static const TraceCoef<T>* stage_tc(const helm_problem* p) {
    if constexpr (sizeof(T) == 8) return p->habc ? p->d_tcid64 : p->d_tc64;
    else return p->habc ? p->d_tcid128 : p->d_tc128;
}
// the matrix an interface stage applies (KMAT_*)
static const void* stage_kmat(const helm_problem* p, int kmat) {
    switch (kmat) {
        case KMAT_LQ: return p->d_Lq;
        case KMAT_D1: return p->d_D1;
        case KMAT_D2: return p->d_D2;
        default: return p->d_K;
    }
}

// event pair around one launch of class k (no-op when profiling is off)
static void prof_begin(helm_problem* p, int k, cudaStream_t st) {
    if (!p->prof_on || p->prof_capture) return;
    auto& q = p->prof[k];
    if (q.used == q.a.size()) {
        cudaEvent_t e1, e2;
        cudaEventCreate(&e1);
        cudaEventCreate(&e2);
        q.a.push_back(e1);
        q.b.push_back(e2);
    }
    cudaEventRecord(q.a[q.used], st);
}
static void prof_end(helm_problem* p, int k, double bytes, cudaStream_t st, double flops = 0.0) {
    if (!p->prof_on) return;
    if (p->prof_capture) {                       // accounting of a sequence being captured
        p->cap_bytes[k] += bytes;
        p->cap_flops[k] += flops;
        p->cap_kernels[k] += 1;
        return;
    }
    auto& q = p->prof[k];
    cudaEventRecord(q.b[q.used], st);
    ++q.used;
    ++q.kernels;
    q.bytes += bytes;
    q.flops += flops;
}
// work known only after the launch (e.g. a pass the device decided to run)
static void prof_add(helm_problem* p, int k, double bytes, double flops) {
    if (!p->prof_on) return;
    p->prof[k].bytes += bytes;
    p->prof[k].flops += flops;
}

extern "C" helm_status helm_profile(helm_problem* p, int on) {
    if (!p) { set_error("helm_profile: NULL handle"); return HELM_ERR_ARG; }
    for (auto& q : p->prof) { q.used = 0; q.kernels = 0; q.bytes = 0; q.flops = 0; }
    p->prof_on = on != 0;
    return HELM_OK;
}

extern "C" helm_status helm_profile_read(helm_problem* p, int k, helm_kstat* out) {
    if (!p || !out || k < 0 || k > 4) { set_error("helm_profile_read: bad argument"); return HELM_ERR_ARG; }
    auto& q = p->prof[k];
    double ms = 0;
    for (size_t i = 0; i < q.used; ++i) {
        cudaError_t e = cudaEventSynchronize(q.b[i]);
        if (e != cudaSuccess) return cuda_status(e, "helm_profile_read");
        float t = 0;
        cudaEventElapsedTime(&t, q.a[i], q.b[i]);
        ms += t;
    }
    out->launches = q.kernels;
    out->ms = ms;
    out->bytes = q.bytes;
    out->flops = q.flops;
    return HELM_OK;
}

// the captured graphs refer to the factors and the workspace: drop them whenever either changes
static void drop_graphs(helm_problem* p) {
    for (auto& g : p->graphs) {
        cudaGraphExecDestroy(g.exec);
        if (g.tmpl) cudaGraphDestroy(g.tmpl);
    }
    p->graphs.clear();
}
static void free_pc_ws(helm_problem* p) {
    drop_graphs(p);
    for (auto& b : p->d_trace) dfree(b);
    dfree(p->d_yws);
    dfree(p->d_escr);
    dfree(p->d_r64);
    dfree(p->d_pc_norm);
    dfree(p->d_pc_partial);
    p->ws_nrhs = 0;
}
static void free_kw(KrylovWS& w) {
    dfree(w.V); dfree(w.Z); dfree(w.H); dfree(w.cs); dfree(w.sn); dfree(w.g);
    dfree(w.h1); dfree(w.h2); dfree(w.hsum); dfree(w.y); dfree(w.cpart);
    dfree(w.rpart); dfree(w.rn); dfree(w.est); dfree(w.invh); dfree(w.active); dfree(w.jcount); dfree(w.need);
    dfree(w.mgs_part); dfree(w.mgs_bar); dfree(w.b); dfree(w.x);
    dfree(w.ctl); dfree(w.iters); dfree(w.thr);
    w.nrhs = w.restart = 0;
    w.n = 0;
}
static void free_krylov(helm_problem* p) {
    free_kw(p->kw);
    free_kw(p->kwi);
}
static void free_adj(helm_problem* p) {
    dfree(p->d_res); dfree(p->d_fadj); dfree(p->d_U); dfree(p->d_L); dfree(p->d_jpart);
    p->aw_nsrc = p->aw_nrec = 0;
}

static constexpr int kPartialBlocks = 1216;   // 8 per SM on 152 SMs

// ------------------------------------------------------------------- setup
extern "C" void helm_default_opts(helm_opts* o) {
    if (!o) return;
    o->restart = 50;
    o->maxit = 1000;
    o->tol = 1e-6;
    o->x0_given = 0;
    o->sched = HELM_SCHED_BSP;
    o->use_graph = 0;
    o->hist = nullptr;
    o->ortho = HELM_ORTHO_MGS;
    o->inner_maxit = 0;
    o->inner_restart = 100;
    o->inner_tol = 1e-4;
    o->persistent = 0;
    o->inner_hist = nullptr;
    o->inner_fp64 = 0;
    o->wait_cycles = 0;
}

extern "C" long long helm_inner_steps(const helm_problem* p) { return p ? p->inner_steps : 0; }
extern "C" void helm_default_setup_opts(helm_setup_opts* o) {
    if (!o) return;
    o->transmission = HELM_TC_OPTIMIZED;
    o->tc_scale = 1.0;
    o->boundary_operators = 1;
    o->tensor_cores = 1;
    o->tc_min_rhs = 16;
    o->autotune = 1;
    o->tc_iface_min_ctas = -1;
    o->device_budget = 0;
    o->n_pade = 8;
    o->pade_phi = 3.14159265358979323846 / 3.0;
    o->tc_factor = 1;
    o->sym_k = 1;
}

extern "C" const char* helm_last_error(void) { return g_err.c_str(); }

extern "C" helm_status helm_schedule_info(int N1, int N2, int sched, int* steps, int* stages) {
    if (N1 < 1 || N2 < 1 || ((sched < 0 || sched >= HELM_NSCHED)))
        return arg_error("helm_schedule_info: N1, N2 >= 1 and a valid schedule are required");
    const int Ng = N1 + N2 - 1;
    std::vector<std::vector<int>> ondiag(Ng + 2);
    std::vector<int> all;
    int id = 0;
    for (int d = 2; d <= Ng + 1; ++d)
        for (int i1 = 1; i1 <= N1; ++i1) {
            const int i2 = d - i1;
            if (i2 >= 1 && i2 <= N2) { ondiag[d].push_back(id); all.push_back(id); ++id; }
        }
    const bool inter = N1 * N2 > 1;
    auto st = build_schedule(sched, N1, N2, ondiag, all, inter);
    if (steps) *steps = inter ? sweep_steps(sched, N1, N2) : 0;
    if (stages) *stages = (int)st.size();
    return HELM_OK;
}

static std::vector<int> make_cuts(int n, int parts, const int* cuts) {
    std::vector<int> c(parts + 1);
    if (cuts) {
        for (int k = 0; k <= parts; ++k) c[k] = cuts[k];
    } else {
        const int q = n / parts, r = n % parts;
        c[0] = 0;
        for (int k = 0; k < parts; ++k) c[k + 1] = c[k] + q + (k < r ? 1 : 0);
    }
    return c;
}

// The HABC transmission's setup (k_habc.cu): per interface slot the side matrix
// Rin = (I - h T / 2)^{-1} (FP64), the identity stage coefficients and the slot-swap
// table.  d_ssub / d_sside / d_slen: the slots' subdomain, side and length on the device.
static helm_status habc_setup(helm_problem* p, const int* d_ssub, const int* d_sside, const int* d_slen,
                              const std::vector<int>& slot_len, const std::vector<int>& slot_off) {
    const int nslots = p->nslots;
    p->slot_len = slot_len;
    for (int k = 0; k < nslots; ++k) p->slot_of_toff[slot_off[k]] = k;
    p->slot_moff.assign(nslots, 0);
    long long tot = 0;
    int max_len = 0;
    for (int k = 0; k < nslots; ++k) {
        p->slot_moff[k] = tot;
        tot += (long long)slot_len[k] * slot_len[k];
        max_len = std::max(max_len, slot_len[k]);
    }
    if (gj_grid(max_len) <= 0 || gj_grid(p->max_Lb) <= 0) {
        set_error("helm_setup: the HABC transmission takes at most 1024 interface boundary points per subdomain");
        return HELM_ERR_UNSUPPORTED;
    }
    helm_status status = HELM_OK;
    double2* Y = nullptr;
    long long* d_moff = nullptr;
    void* d_mats = nullptr;
    double2* pub = nullptr;
    unsigned* bar = nullptr;
    int* info = nullptr;
    do {
        cudaError_t e;
        if ((e = dalloc(p->d_rin, tot)) != cudaSuccess || (e = dalloc(Y, tot)) != cudaSuccess ||
            (e = dalloc(d_moff, nslots)) != cudaSuccess) { status = cuda_status(e, "helm_setup: HABC side matrices"); break; }
        cudaMemcpy(d_moff, p->slot_moff.data(), nslots * sizeof(long long), cudaMemcpyHostToDevice);
        e = launch_habc_sides(p->d_m2, p->nx, p->h, p->omega, p->sopts.n_pade, p->sopts.pade_phi, d_ssub, d_sside,
                              d_slen, d_moff, nslots, max_len, p->d_subtab, p->d_rin, Y, 0);
        if (e != cudaSuccess) { status = cuda_status(e, "helm_setup: HABC side operators"); break; }
        // Rin_s = (I - h T_s / 2)^{-1}, in place
        std::vector<unsigned char> mats(gj_mat_bytes() * nslots);
        for (int k = 0; k < nslots; ++k) gj_mat_fill(mats.data(), k, p->d_rin + p->slot_moff[k], slot_len[k], slot_len[k]);
        if ((e = cudaMalloc(&d_mats, mats.size())) != cudaSuccess || (e = dalloc(pub, 2 * (size_t)(max_len + 2))) ||
            (e = dalloc(bar, 2)) || (e = dalloc(info, nslots))) { status = cuda_status(e, "helm_setup: HABC inversion"); break; }
        cudaMemcpy(d_mats, mats.data(), mats.size(), cudaMemcpyHostToDevice);
        cudaMemset(bar, 0, 2 * sizeof(unsigned));
        cudaMemset(info, 0, nslots * sizeof(int));
        e = launch_gj_inverse(d_mats, nslots, max_len, pub, bar, p->d_err, info, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) { status = cuda_status(e, "helm_setup: HABC side inversion"); break; }
        std::vector<int> hinfo(nslots);
        cudaMemcpy(hinfo.data(), info, nslots * sizeof(int), cudaMemcpyDeviceToHost);
        for (int k = 0; k < nslots; ++k)
            if (hinfo[k]) { set_error("helm_setup: singular HABC side factor I - h T / 2"); status = HELM_ERR_ARG; }
        if (status != HELM_OK) break;
        // stage coefficients: the HABC stages apply their maps in full (cin = 1, ca = 0, cb = 1)
        std::vector<TraceCoef<double2>> id128(p->ntrace, TraceCoef<double2>{make_double2(1, 0), make_double2(0, 0),
                                                                             make_double2(1, 0)});
        std::vector<TraceCoef<float2>> id64(p->ntrace, TraceCoef<float2>{make_float2(1, 0), make_float2(0, 0),
                                                                          make_float2(1, 0)});
        // the point pt of slot (i, j) <-> the point pt of slot (j, i)
        std::vector<int> swp(p->ntrace, 0);
        for (auto& sh : p->subs)
            for (int sd = 0; sd < 4; ++sd) {
                if (sh.dev.tin[sd] < 0) continue;
                const int len = (sd == SW || sd == SE) ? sh.dev.my : sh.dev.mx;
                for (int pt = 0; pt < len; ++pt) swp[sh.dev.tin[sd] + pt] = sh.dev.tout[sd] + pt;
            }
        if ((e = dalloc(p->d_tcid128, p->ntrace)) || (e = dalloc(p->d_tcid64, p->ntrace)) ||
            (e = dalloc(p->d_swap, p->ntrace))) { status = cuda_status(e, "helm_setup: HABC tables"); break; }
        cudaMemcpy(p->d_tcid128, id128.data(), id128.size() * sizeof(id128[0]), cudaMemcpyHostToDevice);
        cudaMemcpy(p->d_tcid64, id64.data(), id64.size() * sizeof(id64[0]), cudaMemcpyHostToDevice);
        if ((e = cudaMemcpy(p->d_swap, swp.data(), swp.size() * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) {
            status = cuda_status(e, "helm_setup: HABC tables");
            break;
        }
    } while (0);
    dfree(Y); dfree(d_moff); dfree(pub); dfree(bar); dfree(info);
    if (d_mats) cudaFree(d_mats);
    if (status == HELM_OK) {
        int v = 0;
        cudaMemcpy(&v, p->d_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (v) {
            cudaMemset(p->d_err, 0, sizeof(int));
            set_error("helm_setup: a device wait timed out in the HABC setup");
            status = HELM_ERR_TIMEOUT;
        }
    }
    p->habc = status == HELM_OK;
    return status;
}

extern "C" helm_status helm_setup(int n_x, int n_y, double h, double omega, const double* m2, int N1, int N2,
                                  const int* xcuts, const int* ycuts, const helm_setup_opts* opts,
                                  helm_problem** out) {
    NvtxRange nvtx("helm_setup");
    if (!out) return arg_error("helm_setup: out is NULL");
    *out = nullptr;
    if (n_x < 1 || n_y < 1) return arg_error("helm_setup: n_x, n_y must be >= 1");
    if (!(h > 0) || !(omega > 0)) return arg_error("helm_setup: h and omega must be > 0");
    if (!m2) return arg_error("helm_setup: m2 is NULL");
    HcCall hcc{{m2, (size_t)n_x * n_y * sizeof(double)}};
    if (N1 < 1 || N2 < 1 || N1 > n_x || N2 > n_y) return arg_error("helm_setup: need 1 <= N1 <= n_x, 1 <= N2 <= n_y");
    helm_setup_opts so;
    helm_default_setup_opts(&so);
    if (opts) so = *opts;
    if (so.transmission != HELM_TC_OPTIMIZED && so.transmission != HELM_TC_IMPEDANCE && so.transmission != HELM_TC_HABC)
        return arg_error("helm_setup: unknown transmission");
    if (so.transmission != HELM_TC_IMPEDANCE && !(so.tc_scale > 0)) return arg_error("helm_setup: tc_scale must be > 0");
    if (so.transmission == HELM_TC_HABC && (so.n_pade < 0 || so.n_pade > 64 || !std::isfinite(so.pade_phi)))
        return arg_error("helm_setup: n_pade must be in 0..64 and pade_phi finite");
    if (so.transmission == HELM_TC_HABC && !so.boundary_operators) {
        set_error("helm_setup: the HABC transmission needs boundary_operators = 1");
        return HELM_ERR_UNSUPPORTED;
    }
    if (so.tensor_cores < 0 || so.tensor_cores > 2) return arg_error("helm_setup: tensor_cores must be 0, 1 or 2");
    if (so.tc_min_rhs < 1) return arg_error("helm_setup: tc_min_rhs must be >= 1");
    if (so.tc_factor != 0 && so.tc_factor != 1) return arg_error("helm_setup: tc_factor must be 0 or 1");
    if (so.autotune != 0 && so.autotune != 1) return arg_error("helm_setup: autotune must be 0 or 1");
    if (so.tc_iface_min_ctas < -1) return arg_error("helm_setup: tc_iface_min_ctas must be >= -1");

    auto xc = make_cuts(n_x, N1, xcuts), yc = make_cuts(n_y, N2, ycuts);
    for (int k = 0; k < N1; ++k)
        if (xc[k + 1] <= xc[k]) return arg_error("helm_setup: xcuts must increase strictly");
    for (int k = 0; k < N2; ++k)
        if (yc[k + 1] <= yc[k]) return arg_error("helm_setup: ycuts must increase strictly");
    if (xc[0] != 0 || xc[N1] != n_x || yc[0] != 0 || yc[N2] != n_y)
        return arg_error("helm_setup: cuts must run from 0 to n");

    helm_problem* p = new (std::nothrow) helm_problem();
    if (!p) { set_error("helm_setup: host allocation failed"); return HELM_ERR_OOM; }
    p->nx = n_x; p->ny = n_y; p->N1 = N1; p->N2 = N2; p->h = h; p->omega = omega; p->sopts = so;
    p->xcut = xc; p->ycut = yc;
    {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            p->num_sms = 1;                     // a later CUDA call reports the failure
    }
    const int Ng = N1 + N2 - 1;

    // subdomains in the paper's order on multi-indices (|i|_1, then i1), Section 2
    std::vector<int> subid(N1 * N2);
    p->ondiag.assign(Ng + 2, {});
    for (int d = 2; d <= Ng + 1; ++d)
        for (int i1 = 1; i1 <= N1; ++i1) {
            const int i2 = d - i1;
            if (i2 < 1 || i2 > N2) continue;
            SubHost s{};
            s.i1 = i1; s.i2 = i2; s.diag = d;
            s.dev.x0 = xc[i1 - 1]; s.dev.mx = xc[i1] - xc[i1 - 1];
            s.dev.y0 = yc[i2 - 1]; s.dev.my = yc[i2] - yc[i2 - 1];
            for (int k = 0; k < 4; ++k) { s.dev.tin[k] = -1; s.dev.tout[k] = -1; }
            const int id = (int)p->subs.size();
            subid[(i2 - 1) * N1 + (i1 - 1)] = id;
            p->ondiag[d].push_back(id);
            p->all.push_back(id);
            p->subs.push_back(s);
            p->max_mx = std::max(p->max_mx, s.dev.mx);
            p->max_my = std::max(p->max_my, s.dev.my);
        }
    if (p->max_mx > 256) { delete p; return arg_error("helm_setup: subdomains wider than 256 nodes are not supported"); }
    long long loff = 0;
    for (auto& s : p->subs) {
        s.dev.loff = loff; s.dev.yoff = loff; loff += (long long)s.dev.mx * s.dev.my;
        s.dev.tcmt = tc_tiles(s.dev.mx);
        s.dev.eoff = p->etot;
        p->etot += 2LL * (s.dev.mx + s.dev.my);
    }

    // interface unknowns (i, j) in the paper's pair order m(i, j) (Section 2)
    std::vector<int> slot_sub, slot_side, slot_off, slot_len;
    auto nb_of = [&](const SubHost& s, int side, int& j1, int& j2) {
        j1 = s.i1 + (side == SE) - (side == SW);
        j2 = s.i2 + (side == SN) - (side == SS);
        return j1 >= 1 && j1 <= N1 && j2 >= 1 && j2 <= N2;
    };
    long long off = 0;
    for (int id = 0; id < (int)p->subs.size(); ++id) {
        auto& s = p->subs[id];
        std::vector<std::pair<std::pair<int, int>, int>> nbs;   // ((|j|_1, j1), side)
        for (int side = 0; side < 4; ++side) {
            int j1, j2;
            if (nb_of(s, side, j1, j2)) nbs.push_back({{j1 + j2, j1}, side});
        }
        std::sort(nbs.begin(), nbs.end());
        for (auto& e : nbs) {
            const int side = e.second;
            const int len = (side == SW || side == SE) ? s.dev.my : s.dev.mx;
            s.dev.tin[side] = (int)off;
            slot_sub.push_back(id); slot_side.push_back(side); slot_off.push_back((int)off); slot_len.push_back(len);
            off += len;
        }
    }
    if (off > (1LL << 30)) { delete p; return arg_error("helm_setup: too many interface unknowns"); }
    p->ntrace = off;
    p->nslots = (int)slot_sub.size();
    for (auto& s : p->subs)
        for (int side = 0; side < 4; ++side) {
            int j1, j2;
            if (!nb_of(s, side, j1, j2)) continue;
            const int opp = side ^ 1;           // W<->E, S<->N
            s.dev.tout[side] = p->subs[subid[(j2 - 1) * N1 + (j1 - 1)]].dev.tin[opp];
        }
    // interface boundary vector (W, E, S, N interface sides) and boundary-operator offsets
    long long koff = 0;
    for (auto& s : p->subs) {
        int lb = 0;
        for (int side = 0; side < 4; ++side) {
            s.dev.bo[side] = -1;
            if (s.dev.tin[side] < 0) continue;
            s.dev.bo[side] = lb;
            lb += (side == SW || side == SE) ? s.dev.my : s.dev.mx;
        }
        s.dev.Lb = lb;
        s.dev.koff = koff;
        koff += (long long)lb * lb;
        s.dev.kpoff = p->kp_elems;
        p->kp_elems += sym_tiles(lb) * SYM_TB * SYM_TB;
        p->max_Lb = std::max(p->max_Lb, lb);
    }
    p->sym_ntmax = (p->max_Lb + SYM_TB - 1) / SYM_TB;

    // stage lists and their subdomain arrays
    std::vector<int> all_stage_subs;
    // a list of subdomains split by tensor-core tile count (1: mx <= 128, 2: mx <= 256)
    auto tc_classes = [&](const std::vector<int>& v, int* off, int* n) {
        for (int c = 0; c < 2; ++c) {
            off[c] = (int)all_stage_subs.size();
            for (int id : v)
                if (p->subs[id].dev.tcmt == c + 1) all_stage_subs.push_back(id);
            n[c] = (int)all_stage_subs.size() - off[c];
        }
    };
    for (int sc = 0; sc < HELM_NSCHED; ++sc) {
        p->sched[sc] = build_schedule(sc, N1, N2, p->ondiag, p->all, p->nslots > 0);
        for (auto& st : p->sched[sc]) {
            st.sub_off = (int)all_stage_subs.size();
            all_stage_subs.insert(all_stage_subs.end(), st.subs.begin(), st.subs.end());
            tc_classes(st.subs, st.tc_off, st.tc_n);
        }
    }
    {
        std::vector<int> ids(p->subs.size());
        for (size_t k = 0; k < ids.size(); ++k) ids[k] = (int)k;
        tc_classes(ids, p->tc_all_off, p->tc_all_n);
    }
    // the interface stages of each schedule (between lifting and reconstruction) for the
    // persistent sweep kernel, when they are all boundary-operator stages
    std::vector<SweepStage> sweep_tab;
    for (int sc = 0; sc < HELM_NSCHED; ++sc) {
        const auto& stg = p->sched[sc];
        p->sweep_off[sc] = (int)sweep_tab.size();
        p->sweep_n[sc] = 0;
        bool all_iface = stg.size() > 2;
        for (size_t i = 1; i + 1 < stg.size(); ++i) all_iface = all_iface && stg[i].iface;
        if (!all_iface) continue;
        for (size_t i = 1; i + 1 < stg.size(); ++i) {
            const StageDesc& sd = stg[i];
            SweepStage t{};
            t.sub_off = sd.sub_off;
            t.nsub = (int)sd.subs.size();
            t.in0 = sd.in0; t.in1 = sd.in1; t.mask = sd.mask;
            t.dst = sd.dst; t.dst2 = sd.dst2; t.base = sd.base; t.sub = sd.sub;
            t.max_rows = 0;
            for (int id : sd.subs) {
                const SubDev& d = p->subs[id].dev;
                int rows = 0;
                for (int sde = 0; sde < 4; ++sde)
                    if ((sd.mask & (1 << sde)) && d.bo[sde] >= 0) rows += (sde == SW || sde == SE) ? d.my : d.mx;
                t.max_rows = std::max(t.max_rows, rows);
            }
            sweep_tab.push_back(t);
        }
        p->sweep_n[sc] = (int)(sweep_tab.size() - p->sweep_off[sc]);
    }
    // dependency-driven sweep tables: per schedule, the work items of its interface
    // stages in order and, per (stage, subdomain), the earlier (stage, subdomain) pairs it
    // must wait for: the last writers of the trace slots it reads and writes and the
    // readers of the slots it overwrites, found by following every slot through the
    // stages (a slot is keyed by its trace offset, per buffer)
    std::vector<int4> dep_items;
    std::vector<int> dep_need, dep_list;
    std::vector<int2> dep_unit;
    for (int sc = 0; sc < HELM_NSCHED; ++sc) {
        p->dep_item_off[sc] = (int)dep_items.size();
        p->dep_unit_off[sc] = (int)dep_need.size();
        if (p->sweep_n[sc] == 0) continue;
        const auto& stg = p->sched[sc];
        std::map<long long, int> lastw[3];
        std::map<long long, std::vector<int>> readers[3];
        for (int si = 0; si < p->sweep_n[sc]; ++si) {
            const StageDesc& sd = stg[si + 1];
            struct Touch { int unit; std::vector<std::pair<int, long long>> reads, writes; };
            std::vector<Touch> touched;
            for (int q = 0; q < (int)sd.subs.size(); ++q) {
                const SubDev& d = p->subs[sd.subs[q]].dev;
                int rows = 0;
                for (int sde = 0; sde < 4; ++sde)
                    if ((sd.mask & (1 << sde)) && d.bo[sde] >= 0) rows += (sde == SW || sde == SE) ? d.my : d.mx;
                const int nblk = (rows + IFACE_RB - 1) / IFACE_RB;
                const int unit = (int)dep_need.size();
                dep_need.push_back(nblk);
                for (int rb = 0; rb < nblk; ++rb) dep_items.push_back(make_int4(si, q, rb, unit));
                Touch t{unit, {}, {}};
                if (nblk > 0) {
                    for (int b : {sd.in0, sd.in1})
                        if (b >= 0)
                            for (int sde = 0; sde < 4; ++sde)
                                if (d.bo[sde] >= 0) t.reads.push_back({b, (long long)d.tin[sde]});
                    for (int sde = 0; sde < 4; ++sde) {
                        if (!((sd.mask & (1 << sde)) && d.bo[sde] >= 0)) continue;
                        for (int b : {sd.base, sd.sub})
                            if (b >= 0) t.reads.push_back({b, (long long)d.tout[sde]});
                        for (int b : {sd.dst, sd.dst2})
                            if (b >= 0) t.writes.push_back({b, (long long)d.tout[sde]});
                    }
                }
                std::vector<int> deps;
                for (auto& r : t.reads) {
                    auto it = lastw[r.first].find(r.second);
                    if (it != lastw[r.first].end()) deps.push_back(it->second);
                }
                for (auto& wr : t.writes) {
                    auto it = lastw[wr.first].find(wr.second);
                    if (it != lastw[wr.first].end()) deps.push_back(it->second);
                    auto jt = readers[wr.first].find(wr.second);
                    if (jt != readers[wr.first].end()) deps.insert(deps.end(), jt->second.begin(), jt->second.end());
                }
                std::sort(deps.begin(), deps.end());
                deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
                dep_unit.push_back(make_int2((int)dep_list.size(), (int)deps.size()));
                dep_list.insert(dep_list.end(), deps.begin(), deps.end());
                touched.push_back(std::move(t));
            }
            // the stage's reads and writes take effect after the whole stage (its items
            // are independent of one another)
            for (auto& t : touched)
                for (auto& r : t.reads) readers[r.first][r.second].push_back(t.unit);
            for (auto& t : touched)
                for (auto& wr : t.writes) {
                    lastw[wr.first][wr.second] = t.unit;
                    readers[wr.first][wr.second].clear();
                }
        }
        p->dep_nitems[sc] = (int)dep_items.size() - p->dep_item_off[sc];
        p->dep_nunits[sc] = (int)dep_need.size() - p->dep_unit_off[sc];
    }

    // device tables
    helm_status status = HELM_OK;
    int *d_xcut = nullptr, *d_ycut = nullptr, *d_subid = nullptr;
    int *d_ssub = nullptr, *d_sside = nullptr, *d_soff = nullptr, *d_slen = nullptr;
    const long long N = p->N();
    auto fail = [&](cudaError_t e, const char* w) {
        status = cuda_status(e, w);
        return status;
    };
    do {
        cudaError_t e;
        if ((e = dalloc(p->d_m2, N)) != cudaSuccess) { fail(e, "alloc m2"); break; }
        if ((e = cudaMemcpy(p->d_m2, m2, N * sizeof(double), cudaMemcpyDefault)) != cudaSuccess) { fail(e, "copy m2"); break; }
        if ((e = dalloc(p->d_adiag, N)) != cudaSuccess) { fail(e, "alloc adiag"); break; }
        if ((e = dalloc(p->d_dloc, N)) != cudaSuccess) { fail(e, "alloc dloc"); break; }
        if ((e = dalloc(p->d_subtab, p->subs.size())) != cudaSuccess) { fail(e, "alloc subtab"); break; }
        std::vector<SubDev> tab;
        for (auto& s : p->subs) tab.push_back(s.dev);
        if ((e = cudaMemcpy(p->d_subtab, tab.data(), tab.size() * sizeof(SubDev), cudaMemcpyHostToDevice)) != cudaSuccess) { fail(e, "copy subtab"); break; }
        if ((e = dalloc(d_xcut, xc.size())) || (e = dalloc(d_ycut, yc.size())) || (e = dalloc(d_subid, subid.size()))) { fail(e, "alloc cuts"); break; }
        cudaMemcpy(d_xcut, xc.data(), xc.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(d_ycut, yc.data(), yc.size() * sizeof(int), cudaMemcpyHostToDevice);
        cudaMemcpy(d_subid, subid.data(), subid.size() * sizeof(int), cudaMemcpyHostToDevice);
        // with the HABC the factored base problem has the optimized Robin condition
        const int base_tr = so.transmission == HELM_TC_HABC ? HELM_TC_OPTIMIZED : so.transmission;
        launch_setup_coeffs(p->d_m2, n_x, n_y, h, omega, d_xcut, d_ycut, N1, N2, d_subid, base_tr, so.tc_scale,
                            p->d_adiag, p->d_dloc, p->d_subtab, 0);
        if (p->nslots > 0) {
            if ((e = dalloc(p->d_tc128, p->ntrace)) || (e = dalloc(p->d_tc64, p->ntrace))) { fail(e, "alloc trace coefficients"); break; }
            if ((e = dalloc(d_ssub, p->nslots)) || (e = dalloc(d_sside, p->nslots)) || (e = dalloc(d_soff, p->nslots)) ||
                (e = dalloc(d_slen, p->nslots))) { fail(e, "alloc slots"); break; }
            cudaMemcpy(d_ssub, slot_sub.data(), p->nslots * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(d_sside, slot_side.data(), p->nslots * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(d_soff, slot_off.data(), p->nslots * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(d_slen, slot_len.data(), p->nslots * sizeof(int), cudaMemcpyHostToDevice);
            launch_trace_coeffs(p->d_m2, n_x, h, omega, base_tr, so.tc_scale, d_ssub, d_sside, d_soff, d_slen,
                                p->nslots, p->d_subtab, p->d_tc128, p->d_tc64, 0);
            if (so.transmission == HELM_TC_HABC) {
                const helm_status hs = habc_setup(p, d_ssub, d_sside, d_slen, slot_len, slot_off);
                if (hs != HELM_OK) { status = hs; break; }
            }
        }
        if ((e = dalloc(p->d_stage_subs, all_stage_subs.size())) != cudaSuccess) { fail(e, "alloc stage lists"); break; }
        if ((e = dalloc(p->d_err, 1)) != cudaSuccess) { fail(e, "alloc status word"); break; }
        if ((e = cudaMemset(p->d_err, 0, sizeof(int))) != cudaSuccess) { fail(e, "clear status word"); break; }
        cudaMemcpy(p->d_stage_subs, all_stage_subs.data(), all_stage_subs.size() * sizeof(int), cudaMemcpyHostToDevice);
        if (!sweep_tab.empty()) {
            if ((e = dalloc(p->d_sweep, sweep_tab.size())) != cudaSuccess) { fail(e, "alloc sweep table"); break; }
            cudaMemcpy(p->d_sweep, sweep_tab.data(), sweep_tab.size() * sizeof(SweepStage), cudaMemcpyHostToDevice);
        }
        if (!dep_items.empty()) {
            if ((e = dalloc(p->d_dep_items, dep_items.size())) != cudaSuccess ||
                (e = dalloc(p->d_dep_need, dep_need.size())) != cudaSuccess ||
                (e = dalloc(p->d_dep_unit, dep_unit.size())) != cudaSuccess ||
                (e = dalloc(p->d_dep_list, std::max<size_t>(1, dep_list.size()))) != cudaSuccess ||
                (e = dalloc(p->d_dep_cnt, dep_need.size())) != cudaSuccess) { fail(e, "alloc sweep dependencies"); break; }
            cudaMemcpy(p->d_dep_items, dep_items.data(), dep_items.size() * sizeof(int4), cudaMemcpyHostToDevice);
            cudaMemcpy(p->d_dep_need, dep_need.data(), dep_need.size() * sizeof(int), cudaMemcpyHostToDevice);
            cudaMemcpy(p->d_dep_unit, dep_unit.data(), dep_unit.size() * sizeof(int2), cudaMemcpyHostToDevice);
            if (!dep_list.empty())
                cudaMemcpy(p->d_dep_list, dep_list.data(), dep_list.size() * sizeof(int), cudaMemcpyHostToDevice);
        }
        if ((e = dalloc(p->d_sweep_bar, 2)) != cudaSuccess) { fail(e, "alloc sweep barrier"); break; }
        if ((e = cudaMemset(p->d_sweep_bar, 0, 2 * sizeof(unsigned))) != cudaSuccess) { fail(e, "clear sweep barrier"); break; }
        if ((e = cudaDeviceSynchronize()) != cudaSuccess) { fail(e, "setup kernels"); break; }
    } while (0);
    dfree(d_xcut); dfree(d_ycut); dfree(d_subid); dfree(d_ssub); dfree(d_sside); dfree(d_soff); dfree(d_slen);
    if (status != HELM_OK) { helm_destroy(p); return status; }
    *out = p;
    return HELM_OK;
}

extern "C" helm_status helm_destroy(helm_problem* p) {
    if (!p) return HELM_OK;
    free_pc_ws(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->cap_ev) cudaEventDestroy(p->cap_ev);
    free_krylov(p);
    free_adj(p);
    dfree(p->d_m2); dfree(p->d_adiag); dfree(p->d_dloc); dfree(p->d_subtab);
    dfree(p->d_tc128); dfree(p->d_tc64); dfree(p->d_stage_subs); dfree(p->d_err);
    dfree(p->d_sweep); dfree(p->d_sweep_bar);
    dfree(p->d_dep_items); dfree(p->d_dep_need); dfree(p->d_dep_unit); dfree(p->d_dep_list); dfree(p->d_dep_cnt);
    for (auto& q : p->prof) {
        for (auto e : q.a) cudaEventDestroy(e);
        for (auto e : q.b) cudaEventDestroy(e);
    }
    if (p->d_X) cudaFree(p->d_X);
    if (p->d_K) cudaFree(p->d_K);
    dfree(p->d_Kp); dfree(p->d_symrt);
    if (p->d_Lq) cudaFree(p->d_Lq);
    if (p->d_D1) cudaFree(p->d_D1);
    if (p->d_D2) cudaFree(p->d_D2);
    dfree(p->d_rin); dfree(p->d_swap); dfree(p->d_tcid128); dfree(p->d_tcid64);
    if (p->d_XT) cudaFree(p->d_XT);
    if (p->d_tcpart) cudaFree(p->d_tcpart);
    if (p->d_tccnt) cudaFree(p->d_tccnt);
    delete p;
    return HELM_OK;
}

extern "C" int helm_factor_on_tensor_cores(const helm_problem* p) { return p && p->factored && p->tc_factor_used; }

extern "C" helm_status helm_problem_info(const helm_problem* p, long long* n_unknowns, int* n_subdomains,
                                         long long* n_trace, long long* factor_bytes) {
    if (!p) return arg_error("helm_problem_info: NULL handle");
    if (n_unknowns) *n_unknowns = p->N();
    if (n_subdomains) *n_subdomains = (int)p->subs.size();
    if (n_trace) *n_trace = p->ntrace;
    if (factor_bytes) *factor_bytes = (long long)p->X_bytes;
    return HELM_OK;
}

// Read and clear the device status word (synchronous).  A kernel sets it when
// one of its bounded waits expired; the work of that launch is then invalid.
static helm_status take_device_status(helm_problem* p, const char* who) {
    int v = 0;
    HELM_CUDA_TRY(cudaMemcpy(&v, p->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (v == 0) return HELM_OK;
    HELM_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int)));
    // a grid barrier that gave up may have left its arrival count behind
    if (p->d_sweep_bar) HELM_CUDA_TRY(cudaMemset(p->d_sweep_bar, 0, 2 * sizeof(unsigned)));
    if (p->kw.mgs_bar) HELM_CUDA_TRY(cudaMemset(p->kw.mgs_bar, 0, 2 * sizeof(unsigned)));
    if (p->kwi.mgs_bar) HELM_CUDA_TRY(cudaMemset(p->kwi.mgs_bar, 0, 2 * sizeof(unsigned)));
    set_error(std::string(who) + ": a device wait timed out; results of this call are invalid");
    return HELM_ERR_TIMEOUT;
}

// ------------------------------------------------------ boundary operators
// K_i = interface-boundary block of A_loc^{-1} for every subdomain: one batched
// multi-RHS block solve per group of `NB` unit data (basis mode of the stage kernel).
template <typename R>
static helm_status build_boundary_operators_t(helm_problem* p, cudaStream_t st) {
    using T = Cx<R>;
    if (p->max_Lb == 0) return HELM_OK;
    long long kel = 0;
    for (auto& s : p->subs) kel += (long long)s.dev.Lb * s.dev.Lb;
    // 16 bytes of padding: the staged interface kernel copies whole 16-byte units, up to
    // 8 bytes past the last row of a complex64 operator
    cudaError_t e = cudaMalloc(&p->d_K, (size_t)kel * sizeof(T) + 16);
    if (e != cudaSuccess) { p->d_K = nullptr; return cuda_status(e, "precond_factor: allocating boundary operators"); }
    p->K_bytes = (size_t)kel * sizeof(T);
    const int NB = 64;
    void* yws = nullptr;
    e = cudaMalloc(&yws, (size_t)p->N() * NB * sizeof(T));
    if (e != cudaSuccess) return cuda_status(e, "precond_factor: allocating the basis workspace");
    StageArgs<R> a{};
    a.subtab = p->d_subtab;
    a.nx = p->nx; a.ny = p->ny;
    a.nrhs = NB;
    a.wstride = p->N();
    a.X = (const T*)p->d_X;
    a.tc = sizeof(R) == 4 ? (const TraceCoef<T>*)p->d_tc64 : (const TraceCoef<T>*)p->d_tc128;
    a.yws = (T*)yws;
    a.K = (T*)p->d_K;
    a.err = p->d_err;
    for (int c0 = 0; c0 < p->max_Lb && e == cudaSuccess; c0 += NB) {
        a.col0 = c0;
        if constexpr (sizeof(R) == 4) {
            if (p->d_XT) {
                for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
                    a.subs = p->d_stage_subs + p->tc_all_off[c];
                    e = launch_tc_basis(a, p->d_XT, c + 1, p->tc_split, p->tc_all_n[c], NB, st);
                }
                continue;
            }
        }
        e = launch_basis<R>(a, (int)p->subs.size(), NB, p->max_mx, p->max_my, p->max_w, p->max_ld, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(yws);
    if (e != cudaSuccess) return cuda_status(e, "precond_factor: boundary operators");
    const helm_status ds = take_device_status(p, "precond_factor");
    if (ds != HELM_OK) return ds;
    return HELM_OK;
}

static helm_status build_boundary_operators(helm_problem* p, cudaStream_t st) {
    NvtxRange nvtx("boundary operators");
    return p->prec == HELM_PREC_C64 ? build_boundary_operators_t<float>(p, st)
                                    : build_boundary_operators_t<double>(p, st);
}

// The HABC stage matrices of every subdomain from its base boundary operator K (the
// block comment of k_habc.cu has the algebra), in FP64, in batches of subdomains:
//   KR = K Rin, W = (I - 2 KR + K + K diag(c0))^{-1} = (I - K C)^{-1}, P1 = W KR,
//   RP = Rin P1, RW = Rin W, then Q (replaces K), Lq, D1, D2 in the factor precision.
template <typename R>
static helm_status habc_precompute_t(helm_problem* p, cudaStream_t st) {
    using T = Cx<R>;
    const int nsub = (int)p->subs.size();
    const long long Lb2 = (long long)p->max_Lb * p->max_Lb;
    long long kel = 0;
    for (auto& sh : p->subs) kel += (long long)sh.dev.Lb * sh.dev.Lb;
    // six FP64 temporaries per subdomain of a batch, at most ~2 GB
    const int bsz = (int)std::max<long long>(1, std::min<long long>(nsub, (2LL << 30) / (6 * Lb2 * 16)));
    helm_status status = HELM_OK;
    double2* tmp = nullptr;
    void *Q = nullptr, *Lq = nullptr, *D1 = nullptr, *D2 = nullptr;
    void *d_subs = nullptr, *d_mats = nullptr, *d_gemm = nullptr;
    double2* pub = nullptr;
    unsigned* bar = nullptr;
    int* info = nullptr;
    const size_t mbytes = (size_t)kel * sizeof(T) + 16;     // as K: 16 bytes of padding
    do {
        cudaError_t e;
        if ((e = cudaMalloc(&Q, mbytes)) || (e = cudaMalloc(&Lq, mbytes)) || (e = cudaMalloc(&D1, mbytes)) ||
            (e = cudaMalloc(&D2, mbytes))) { status = cuda_status(e, "precond_factor: HABC stage matrices"); break; }
        if ((e = dalloc(tmp, (size_t)6 * bsz * Lb2)) != cudaSuccess) {
            status = cuda_status(e, "precond_factor: HABC workspace");
            break;
        }
        const int maxprob = std::max(1, 4 * bsz);
        if ((e = cudaMalloc(&d_subs, habc_sub_bytes() * bsz)) || (e = cudaMalloc(&d_mats, gj_mat_bytes() * bsz)) ||
            (e = cudaMalloc(&d_gemm, gemm_prob_bytes() * maxprob)) || (e = dalloc(pub, 2 * (size_t)(p->max_Lb + 2))) ||
            (e = dalloc(bar, 2)) || (e = dalloc(info, bsz))) {
            status = cuda_status(e, "precond_factor: HABC tables");
            break;
        }
        cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
        double2* K64 = tmp;
        double2* KR = tmp + (size_t)bsz * Lb2;
        double2* W = tmp + 2 * (size_t)bsz * Lb2;
        double2* P1 = tmp + 3 * (size_t)bsz * Lb2;
        double2* RP = tmp + 4 * (size_t)bsz * Lb2;
        double2* RW = tmp + 5 * (size_t)bsz * Lb2;
        std::vector<unsigned char> hs(habc_sub_bytes() * bsz), hm(gj_mat_bytes() * bsz), hg(gemm_prob_bytes() * maxprob);
        const double2 one = make_double2(1.0, 0.0);
        for (int b0 = 0; b0 < nsub && status == HELM_OK; b0 += bsz) {
            const int nb = std::min(bsz, nsub - b0);
            // per subdomain: boundary layout, the side matrices of its slots (slot_of_toff:
            // the slot whose trace starts at a given offset), its matrix to invert
            for (int q = 0; q < nb; ++q) {
                const SubDev& d = p->subs[b0 + q].dev;
                int len[4];
                long long moff[4];
                for (int sd = 0; sd < 4; ++sd) {
                    len[sd] = d.bo[sd] >= 0 ? ((sd == SW || sd == SE) ? d.my : d.mx) : 0;
                    moff[sd] = d.tin[sd] >= 0 ? p->slot_moff[p->slot_of_toff.at(d.tin[sd])] : 0;
                }
                habc_sub_fill(hs.data(), q, d.koff, (long long)q * Lb2, d.Lb, d.bo, len, moff, d.tin);
                gj_mat_fill(hm.data(), q, W + (size_t)q * Lb2, d.Lb, d.Lb);
            }
            cudaMemcpyAsync(d_subs, hs.data(), habc_sub_bytes() * nb, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(d_mats, hm.data(), gj_mat_bytes() * nb, cudaMemcpyHostToDevice, st);
            // K in FP64
            e = launch_habc_form<T>(d_subs, nb, p->max_Lb, (const T*)p->d_K, p->d_tc128, K64, KR, W, 0, st);
            // KR = K Rin: per side s, columns [bo_s, bo_s + L) of K times Rin_s
            auto side_products = [&](bool left, const double2* X, double2* out) -> cudaError_t {
                int np = 0, mm = 0, mn = 0;
                for (int q = 0; q < nb; ++q) {
                    const SubDev& d = p->subs[b0 + q].dev;
                    for (int sd = 0; sd < 4; ++sd) {
                        if (d.bo[sd] < 0) continue;
                        const int L = (sd == SW || sd == SE) ? d.my : d.mx;
                        const double2* rin = p->d_rin + p->slot_moff[p->slot_of_toff.at(d.tin[sd])];
                        const size_t t = (size_t)q * Lb2;
                        if (!left)   // out[:, bo + c] = X[:, bo + c'] Rin[c', c]
                            gemm_prob_fill(hg.data(), np++, X + t + d.bo[sd], rin, out + t + d.bo[sd], d.Lb, L, L,
                                           d.Lb, L, d.Lb, one, 0);
                        else         // out[bo + r, :] = Rin[r, r'] X[bo + r', :]
                            gemm_prob_fill(hg.data(), np++, rin, X + t + (size_t)d.bo[sd] * d.Lb,
                                           out + t + (size_t)d.bo[sd] * d.Lb, L, d.Lb, L, L, d.Lb, d.Lb, one, 0);
                        mm = std::max(mm, left ? L : d.Lb);
                        mn = std::max(mn, left ? d.Lb : L);
                    }
                }
                cudaError_t e2 = cudaMemcpyAsync(d_gemm, hg.data(), gemm_prob_bytes() * np, cudaMemcpyHostToDevice, st);
                if (e2 == cudaSuccess) e2 = launch_zgemm_batched(d_gemm, np, mm, mn, st);
                // the host table is reused by the next call: wait for the copy
                if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(st);
                return e2;
            };
            if (e == cudaSuccess) e = side_products(false, K64, KR);
            // W = I - K C, then its inverse in place
            if (e == cudaSuccess) e = launch_habc_form<T>(d_subs, nb, p->max_Lb, (const T*)p->d_K, p->d_tc128, K64, KR, W, 1, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(info, 0, nb * sizeof(int), st);
            if (e == cudaSuccess) e = launch_gj_inverse(d_mats, nb, p->max_Lb, pub, bar, p->d_err, info, st);
            // P1 = W KR
            if (e == cudaSuccess) {
                for (int q = 0; q < nb; ++q) {
                    const SubDev& d = p->subs[b0 + q].dev;
                    const size_t t = (size_t)q * Lb2;
                    gemm_prob_fill(hg.data(), q, W + t, KR + t, P1 + t, d.Lb, d.Lb, d.Lb, d.Lb, d.Lb, d.Lb, one, 0);
                }
                e = cudaMemcpyAsync(d_gemm, hg.data(), gemm_prob_bytes() * nb, cudaMemcpyHostToDevice, st);
                if (e == cudaSuccess) e = launch_zgemm_batched(d_gemm, nb, p->max_Lb, p->max_Lb, st);
                if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            }
            if (e == cudaSuccess) e = side_products(true, P1, RP);
            if (e == cudaSuccess) e = side_products(true, W, RW);
            if (e == cudaSuccess)
                e = launch_habc_final<T>(d_subs, nb, p->max_Lb, p->d_rin, p->d_tc128, P1, RP, W, RW, (T*)Q, (T*)Lq,
                                         (T*)D1, (T*)D2, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) { status = cuda_status(e, "precond_factor: HABC stage matrices"); break; }
            std::vector<int> hinfo(nb);
            cudaMemcpy(hinfo.data(), info, nb * sizeof(int), cudaMemcpyDeviceToHost);
            for (int q = 0; q < nb; ++q)
                if (hinfo[q]) {
                    char buf[160];
                    snprintf(buf, sizeof buf, "precond_factor: I - K C of subdomain %d is singular (pivot %d)", b0 + q,
                             hinfo[q] - 1);
                    set_error(buf);
                    status = HELM_ERR_ARG;
                }
        }
    } while (0);
    dfree(tmp); dfree(pub); dfree(bar); dfree(info);
    if (d_subs) cudaFree(d_subs);
    if (d_mats) cudaFree(d_mats);
    if (d_gemm) cudaFree(d_gemm);
    if (status == HELM_OK) status = take_device_status(p, "precond_factor (HABC stage matrices)");
    if (status != HELM_OK) {
        for (void* q : {Q, Lq, D1, D2}) if (q) cudaFree(q);
        return status;
    }
    // the interface stages apply Q in place of K
    cudaFree(p->d_K);
    p->d_K = Q;
    p->K_bytes *= 4;                 // Q, Lq, D1, D2
    p->d_Lq = Lq;
    p->d_D1 = D1;
    p->d_D2 = D2;
    return HELM_OK;
}
static helm_status habc_precompute(helm_problem* p, cudaStream_t st) {
    NvtxRange nvtx("HABC stage matrices");
    if (p->max_Lb == 0) return HELM_OK;
    return p->prec == HELM_PREC_C64 ? habc_precompute_t<float>(p, st) : habc_precompute_t<double>(p, st);
}

// ----------------------------------------------------------------- factor
// the packed symmetric operators: complex64, the scalar transmissions (the HABC stage
// matrices are not symmetric), K built, at most SYM_MAXLB boundary points per subdomain
static bool sym_wanted(const helm_problem* p, int prec) {
    return p->sopts.sym_k && prec == HELM_PREC_C64 && p->sopts.boundary_operators && !p->habc &&
           p->max_Lb > 0 && p->max_Lb <= SYM_MAXLB;
}
// their bytes: the tiles and the row-tile list
static size_t sym_bytes(const helm_problem* p) {
    return (size_t)p->kp_elems * sizeof(float2) + p->subs.size() * (size_t)p->sym_ntmax * sizeof(int2);
}
static helm_status build_symmetric_operators(helm_problem* p, cudaStream_t st) {
    const size_t ns = p->subs.size();
    std::vector<int2> rt;
    for (size_t i = 0; i < ns; ++i)
        for (int I = 0; I < (p->subs[i].dev.Lb + SYM_TB - 1) / SYM_TB; ++I) rt.push_back(make_int2((int)i, I));
    cudaError_t e;
    if ((e = dalloc(p->d_Kp, (size_t)p->kp_elems)) != cudaSuccess || (e = dalloc(p->d_symrt, rt.size()))) {
        dfree(p->d_Kp); dfree(p->d_symrt);
        return cuda_status(e, "precond_factor: allocating the packed symmetric boundary operators");
    }
    p->sym_nrt = (int)rt.size();
    e = cudaMemcpyAsync(p->d_symrt, rt.data(), rt.size() * sizeof(int2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = launch_sym_pack(p->d_subtab, (int)ns, p->sym_ntmax, (const float2*)p->d_K, p->d_Kp, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "precond_factor: packing the symmetric boundary operators");
    return HELM_OK;
}

extern "C" int helm_iface_symmetric(const helm_problem* p, int nrhs) {
    return p && p->factored && p->d_Kp && nrhs == 1;
}

extern "C" helm_status precond_factor(helm_problem* p, helm_prec prec, void* stream) {
    NvtxRange nvtx("precond_factor");
    if (!p) return arg_error("precond_factor: NULL handle");
    if (prec != HELM_PREC_C128 && prec != HELM_PREC_C64) return arg_error("precond_factor: unknown precision");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t elem = prec == HELM_PREC_C64 ? sizeof(float2) : sizeof(double2);
    // layout of the stored X_r: per subdomain my blocks, each two column halves of
    // widths w0 = mx/2 rounded up to even and mx - w0, leading dimensions even for
    // complex64 so that every half, block and row chunk starts on a 16-byte boundary
    long long xoff = 0, xtoff = 0;
    // second copy for the tensor cores: complex64, enabled, subdomains at most 256 nodes wide
    const int mt = (prec == HELM_PREC_C64 && p->sopts.tensor_cores) ? tc_tiles(p->max_mx) : 0;
    const int split = p->sopts.tensor_cores == 2 ? 1 : 3;
    std::vector<SubDev> tab;
    p->max_w = p->max_ld = 0;
    for (auto& s : p->subs) {
        const int mx = s.dev.mx;
        const int w0 = std::min(mx, ((mx + 1) / 2 + 1) & ~1);
        const int w1 = mx - w0;
        s.dev.w0 = w0;
        s.dev.ld0 = w0;                                                   // even (or mx itself when mx <= 2)
        s.dev.ld1 = prec == HELM_PREC_C64 ? ((w1 + 1) & ~1) : w1;
        if (prec == HELM_PREC_C64 && (s.dev.ld0 & 1)) s.dev.ld0 += 1;
        s.dev.xoff = xoff;
        xoff += (long long)s.dev.my * mx * (s.dev.ld0 + s.dev.ld1);
        s.dev.xtoff = xtoff;
        if (mt) xtoff += tc_layout_floats(mx, s.dev.my, s.dev.tcmt, split);
        p->max_w = std::max(p->max_w, std::max(w0, w1));
        p->max_ld = std::max(p->max_ld, std::max(s.dev.ld0, s.dev.ld1));
        tab.push_back(s.dev);
    }
    const size_t bytes = (size_t)xoff * elem;
    if (p->sopts.device_budget > 0) {
        // the arrays this factorisation keeps: factors, their tensor-core copy, boundary operators
        long long kel = 0;
        for (auto& s : p->subs) kel += (long long)s.dev.Lb * s.dev.Lb;
        const size_t keep = bytes + (size_t)xtoff * sizeof(float) +
                            (p->sopts.boundary_operators ? (size_t)kel * elem * (p->habc ? 4 : 1) : 0) +
                            (sym_wanted(p, prec) ? sym_bytes(p) : 0);
        if (keep > p->sopts.device_budget) {
            char buf[200];
            snprintf(buf, sizeof buf, "precond_factor: the factors need %zu bytes, more than the device budget of %zu",
                     keep, p->sopts.device_budget);
            set_error(buf);
            return HELM_ERR_OOM;
        }
    }
    HELM_CUDA_TRY(cudaStreamSynchronize(st));
    drop_graphs(p);
    if (p->d_X) { cudaFree(p->d_X); p->d_X = nullptr; p->X_bytes = 0; p->factored = 0; }
    if (p->d_K) { cudaFree(p->d_K); p->d_K = nullptr; p->K_bytes = 0; }
    dfree(p->d_Kp); dfree(p->d_symrt);
    for (void** q : {&p->d_Lq, &p->d_D1, &p->d_D2})
        if (*q) { cudaFree(*q); *q = nullptr; }
    if (p->d_XT) { cudaFree(p->d_XT); p->d_XT = nullptr; p->XT_bytes = 0; p->tc_mt = 0; p->tc_split = 0; }
    cudaError_t e = cudaMalloc(&p->d_X, bytes);
    if (e != cudaSuccess) { p->d_X = nullptr; return cuda_status(e, "precond_factor: allocating the factors"); }
    p->X_bytes = bytes;
    HELM_CUDA_TRY(cudaMemcpy(p->d_subtab, tab.data(), tab.size() * sizeof(SubDev), cudaMemcpyHostToDevice));
    const size_t wel = factor_work_elems(p->max_mx, elem);
    void* work = nullptr;
    int* info = nullptr;
    if (wel) {
        e = cudaMalloc(&work, wel * elem * p->subs.size());
        if (e != cudaSuccess) return cuda_status(e, "precond_factor: allocating the factor workspace");
    }
    e = cudaMalloc(&info, p->subs.size() * sizeof(int));
    if (e != cudaSuccess) { if (work) cudaFree(work); return cuda_status(e, "precond_factor: alloc info"); }
    // complex64 with subdomains at most 128 nodes wide: the Gauss-Jordan trailing updates on
    // the tensor cores (k_tc.cu), else the CUDA-core kernel (k_factor.cu)
    p->tc_factor_used = prec == HELM_PREC_C64 && p->sopts.tensor_cores && p->sopts.tc_factor && p->max_mx <= 128;
    if (p->tc_factor_used)
        e = launch_tc_factor(p->d_subtab, (int)p->subs.size(), p->d_dloc, (float2*)p->d_X, info, p->d_err, st);
    else if (prec == HELM_PREC_C64)
        e = launch_factor<float>(p->d_subtab, (int)p->subs.size(), p->max_mx, p->d_dloc, (float2*)p->d_X, (float2*)work,
                                 wel, info, st);
    else
        e = launch_factor<double>(p->d_subtab, (int)p->subs.size(), p->max_mx, p->d_dloc, (double2*)p->d_X,
                                  (double2*)work, wel, info, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    std::vector<int> hinfo(p->subs.size());
    if (e == cudaSuccess) e = cudaMemcpy(hinfo.data(), info, hinfo.size() * sizeof(int), cudaMemcpyDeviceToHost);
    if (work) cudaFree(work);
    cudaFree(info);
    if (e != cudaSuccess) return cuda_status(e, "precond_factor: factor kernel");
    {
        const helm_status ds = take_device_status(p, "precond_factor");
        if (ds != HELM_OK) return ds;
    }
    for (size_t k = 0; k < hinfo.size(); ++k)
        if (hinfo[k]) {
            char buf[160];
            snprintf(buf, sizeof buf, "precond_factor: zero pivot in subdomain %zu (row %d, column %d)", k,
                     (hinfo[k] - 1) / p->subs[k].dev.mx, (hinfo[k] - 1) % p->subs[k].dev.mx);
            set_error(buf);
            return HELM_ERR_ARG;
        }
    p->prec = prec;
    if (mt) {
        e = cudaMalloc(&p->d_XT, (size_t)xtoff * sizeof(float));
        if (e != cudaSuccess) { p->d_XT = nullptr; return cuda_status(e, "precond_factor: allocating the tensor-core factors"); }
        p->XT_bytes = (size_t)xtoff * sizeof(float);
        p->tc_mt = mt;
        p->tc_split = split;
        e = launch_tc_layout(p->d_subtab, (int)p->subs.size(), split, (const float2*)p->d_X, p->d_XT, st);
        if (e != cudaSuccess) return cuda_status(e, "precond_factor: tensor-core layout");
        if (!p->d_tcpart) {
            // a split tensor-core interface stage makes fewer than 4 CTAs per SM, each with
            // 128 rows x 2 x 32 partial sums; fewer than 2 tiles per SM are split
            const long long cap = 4LL * p->num_sms * 128 * 64;
            e = cudaMalloc(&p->d_tcpart, (size_t)cap * sizeof(float));
            if (e == cudaSuccess) e = cudaMalloc(&p->d_tccnt, (size_t)4 * p->num_sms * sizeof(int));
            if (e != cudaSuccess) return cuda_status(e, "precond_factor: allocating the interface-stage scratch");
            p->tcpart_cap = cap;
            p->tccnt_cap = 4 * p->num_sms;
        }
        // the arrival counters start at zero; each factorisation resets them (after a
        // HELM_ERR_TIMEOUT a split tile may have left its counter short of S)
        e = cudaMemsetAsync(p->d_tccnt, 0, (size_t)p->tccnt_cap * sizeof(int), st);
        if (e != cudaSuccess) return cuda_status(e, "precond_factor: resetting the interface-stage counters");
    }
    {
        helm_status ks = p->sopts.boundary_operators ? build_boundary_operators(p, st) : HELM_OK;
        if (ks == HELM_OK && p->habc) ks = habc_precompute(p, st);
        if (ks == HELM_OK && sym_wanted(p, prec)) ks = build_symmetric_operators(p, st);
        if (ks != HELM_OK) return ks;
    }
    p->factored = 1;
    // the workspace depends on the precision
    free_pc_ws(p);
    return HELM_OK;
}

// ------------------------------------------------------------ preconditioner
// stages over nrhs right-hand sides run on the tensor cores
static bool tc_used(const helm_problem* p, int nrhs) {
    return p->d_XT != nullptr && nrhs >= std::max(1, p->sopts.tc_min_rhs);
}

static helm_status ensure_pc_ws(helm_problem* p, int nrhs) {
    if (p->ws_nrhs >= nrhs) return HELM_OK;
    free_pc_ws(p);
    const size_t elem = p->prec == HELM_PREC_C64 ? sizeof(float2) : sizeof(double2);
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < (p->habc ? 4 : 3) && e == cudaSuccess && p->ntrace > 0; ++b)
        e = cudaMalloc(&p->d_trace[b], (size_t)p->ntrace * nrhs * elem);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_yws, (size_t)p->N() * nrhs * elem);
    if (e == cudaSuccess && tc_used(p, nrhs)) {
        e = cudaMalloc(&p->d_escr, (size_t)2 * p->etot * nrhs * sizeof(float2));
        if (e == cudaSuccess) e = cudaMalloc(&p->d_r64, (size_t)p->N() * nrhs * sizeof(float2));
    }
    if (e == cudaSuccess) e = dalloc(p->d_pc_norm, 3 * (size_t)nrhs);
    if (e == cudaSuccess) e = dalloc(p->d_pc_partial, (size_t)kPartialBlocks * nrhs);
    if (e != cudaSuccess) { free_pc_ws(p); return cuda_status(e, "allocating the preconditioner workspace"); }
    p->ws_nrhs = nrhs;
    return HELM_OK;
}

// scratch of one preconditioner application: three interface buffers of
// ntrace*nrhs values, the solve workspace (N*nrhs), 3*nrhs norms and
// kPartialBlocks*nrhs partial sums
struct PcWork {
    void* trace[4];                  // B, X, Y (and U with the HABC transmission)
    void* yws;
    double* norm;
    double* partial;
    void* escr;                      // tensor-core path only (else null)
    void* r64;
};

// algorithmic bytes and flops of one interface stage: the rows of K it applies,
// the incoming data it reads, the outgoing data (and base / sub) it moves
// (packed symmetric form: the stored tiles the stage reads, each once, instead of the rows)
static void iface_accounting(const helm_problem* p, const StageDesc& sd, int nrhs, double sT, double& bytes,
                             double& flops, bool sym = false) {
    for (int id : sd.subs) {
        const SubDev& d = p->subs[id].dev;
        double rows = 0;
        for (int sde = 0; sde < 4; ++sde)
            if ((sd.mask & (1 << sde)) && d.bo[sde] >= 0) rows += (sde == SW || sde == SE) ? d.my : d.mx;
        const double io = d.Lb * sT * ((sd.in0 >= 0) + (sd.in1 >= 0)) +
                          rows * sT * (1 + (sd.dst2 >= 0) + (sd.base >= 0) + (sd.sub >= 0));
        double kbytes = rows * d.Lb * sT;
        if (sym) {
            const int nt = (d.Lb + SYM_TB - 1) / SYM_TB;
            unsigned long long M = 0;
            for (int sde = 0; sde < 4; ++sde)
                if ((sd.mask & (1 << sde)) && d.bo[sde] >= 0) {
                    const int len = (sde == SW || sde == SE) ? d.my : d.mx;
                    for (int t = d.bo[sde] / SYM_TB; t <= (d.bo[sde] + len - 1) / SYM_TB; ++t) M |= 1ull << t;
                }
            long long tiles = 0;
            for (int I = 0; I < nt; ++I)
                for (int J = I; J < nt; ++J) tiles += ((M >> I) & 1) || ((M >> J) & 1);
            kbytes = (double)tiles * SYM_TB * SYM_TB * sT;
        }
        bytes += kbytes + io * nrhs;
        flops += 8.0 * rows * d.Lb * nrhs;
    }
}

// The interface stages of a schedule (all but the lifting and the reconstruction)
// in the persistent sweep kernel; false when it does not apply (no boundary
// operators, or no cooperative launch), and the caller runs the stages one by one.
template <typename R>
static bool run_sweep_persistent(helm_problem* p, const PcWork& w, int sched, int nrhs, cudaStream_t st,
                                 helm_status& status) {
    using T = Cx<R>;
    if (!p->persistent || !p->d_K || !p->d_sweep || p->sweep_n[sched] == 0) return false;
    const int grid = p->persistent == 1 ? sweep_grid<R>(nrhs, p->max_Lb) : 1;
    if (grid <= 0) return false;
    if (p->persistent == 2 && p->dep_nitems[sched] == 0) return false;
    IfaceArgs<R> a{};
    a.subtab = p->d_subtab;
    a.subs = p->d_stage_subs;
    a.nrhs = nrhs;
    a.ntrace = p->ntrace;
    a.K = (const T*)p->d_K;
    a.tc = stage_tc<T>(p);
    for (int b = 0; b < 3; ++b) a.bufs[b] = w.trace[b];
    a.err = p->d_err;
    double bytes = 0, flops = 0;
    if (p->prof_on) {
        const auto& stg = p->sched[sched];
        for (size_t i = 1; i + 1 < stg.size(); ++i) iface_accounting(p, stg[i], nrhs, sizeof(T), bytes, flops);
    }
    prof_begin(p, HELM_K_TRACE, st);
    cudaError_t e;
    if (p->persistent == 2) {
        // dependency-driven: the counters of this schedule start at zero
        e = cudaMemsetAsync(p->d_dep_cnt + p->dep_unit_off[sched], 0, (size_t)p->dep_nunits[sched] * sizeof(int), st);
        if (e == cudaSuccess)
            e = launch_sweep_dep<R>(a, p->d_sweep + p->sweep_off[sched], p->d_dep_items + p->dep_item_off[sched],
                                    p->dep_nitems[sched], p->d_dep_need, p->d_dep_unit, p->d_dep_list, p->d_dep_cnt,
                                    p->max_Lb, st);
    } else {
        e = launch_sweep<R>(a, p->d_sweep + p->sweep_off[sched], p->sweep_n[sched], p->max_Lb, grid, p->d_sweep_bar,
                            p->d_err, st);
    }
    prof_end(p, HELM_K_TRACE, bytes, st, flops);
    if (p->prof_on && !p->prof_capture) p->prof[HELM_K_TRACE].kernels += p->sweep_n[sched] - 1;
    status = e == cudaSuccess ? HELM_OK : cuda_status(e, "sweep kernel launch");
    return true;
}

// per-application constants of the preconditioner
struct PcCtx {
    const double* rinv = nullptr;    // complex64: 1/||r|| per RHS (the source is scaled to unit norm)
    const double* rsc = nullptr;     // complex64: ||r|| per RHS (applied to the output)
    bool tc = false;                 // the stages run on the tensor cores
};

template <typename R>
static PcCtx precond_prologue(helm_problem* p, const PcWork& w, const double2* r, int nrhs, cudaStream_t st) {
    PcCtx cx;
    if (sizeof(R) == 4) {
        // scale each right-hand side to unit 2-norm before rounding to complex64
        launch_norm2_partial(r, p->N(), nrhs, p->N(), w.partial, kPartialBlocks, st);
        launch_reduce_rows(w.partial, kPartialBlocks, nrhs, w.norm, 0, st);
        launch_scale_from_norm(w.norm, w.norm + nrhs, w.norm + 2 * nrhs, nrhs, st);
        cx.rinv = w.norm + nrhs;
        cx.rsc = w.norm + 2 * nrhs;
    }
    // the tensor-core stages read the scaled source in complex64
    cx.tc = sizeof(R) == 4 && tc_used(p, nrhs) && w.escr && w.r64;
    if (cx.tc) launch_to_c64_scaled(r, cx.rinv, (float2*)w.r64, p->N(), nrhs, st);
    return cx;
}

// one stage of a schedule (one batched launch, two for mixed tensor-core tile counts)
// autotuned launch shape of the interface stages for nrhs RHS (nullptr: the fixed rules)
static const IfaceCfg* tuned_shape(const helm_problem* p, int nrhs) {
    for (const auto& t : p->iface_tuned)
        if (t.prec == p->prec && t.nrhs == nrhs) return &t.cfg;
    return nullptr;
}
// the tensor-core form of the interface stages for nrhs RHS, where it is allowed
static bool iface_tc_cfg(const helm_problem* p, int nrhs, IfaceCfg& c) {
    if (p->prec != HELM_PREC_C64 || !tc_used(p, nrhs) || (p->tc_split != 1 && p->tc_split != 3)) return false;
    c = IfaceCfg{};
    c.nr = nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1;
    c.tc = p->tc_split;
    c.tc_nb = nrhs >= 32 ? 32 : 16;
    c.tc_min_ctas = p->sopts.tc_iface_min_ctas;
    return true;
}
// the launch shape the interface stages use: the autotuned one, else the tensor cores
// where allowed, else the kernel's fixed rules (nullptr)
static const IfaceCfg* iface_shape_for(const helm_problem* p, int nrhs, IfaceCfg& tmp) {
    if (const IfaceCfg* t = tuned_shape(p, nrhs)) return t;
    if (iface_tc_cfg(p, nrhs, tmp)) return &tmp;
    return nullptr;
}

// The autotuner of the interface-stage kernel: the first application with nrhs >= 2 RHS
// times each candidate shape (RHS per block 2/4/8/16 up to nrhs, K staged or not) on
// the stage S (every subdomain, every side: reads X, writes B, so it may run any number
// of times) with CUDA events on the caller's stream, after the work already queued
// there, and keeps the fastest.  Runs before any graph capture of that RHS count.
template <typename R>
static helm_status tune_shape_t(helm_problem* p, int nrhs, cudaStream_t st) {
    using T = Cx<R>;
    const StageDesc& all = p->sched[HELM_SCHED_BSP].front();
    IfaceArgs<R> ia{};
    ia.subtab = p->d_subtab;
    ia.subs = p->d_stage_subs + all.sub_off;
    ia.nrhs = nrhs;
    ia.ntrace = p->ntrace;
    ia.K = (const T*)p->d_K;
    ia.tc = stage_tc<T>(p);
    ia.gin0 = (const T*)p->d_trace[BUF_X];
    ia.mask = 15;
    ia.dst = (T*)p->d_trace[BUF_B];
    ia.sub = (const T*)p->d_trace[BUF_X];
    ia.err = p->d_err;
    ia.part = p->d_tcpart; ia.part_cap = p->tcpart_cap;
    ia.cnt = p->d_tccnt; ia.cnt_cap = p->tccnt_cap;
    int max_rows = 0;
    for (int id : all.subs) {
        const SubDev& d = p->subs[id].dev;
        int rows = 0;
        for (int sde = 0; sde < 4; ++sde)
            if (d.bo[sde] >= 0) rows += (sde == SW || sde == SE) ? d.my : d.mx;
        max_rows = std::max(max_rows, rows);
    }
    HELM_CUDA_TRY(cudaMemsetAsync(p->d_trace[BUF_X], 0, (size_t)p->ntrace * nrhs * sizeof(T), st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HELM_CUDA_TRY(cudaEventCreate(&e0));
    HELM_CUDA_TRY(cudaEventCreate(&e1));
    const long long before = helm_launch_count();
    IfaceCfg best{};
    float best_ms = 1e30f;
    // candidates: CUDA cores with 2..16 RHS per block, K staged or not; the tensor-core
    // form with 16 or 32 RHS per CTA where it is allowed
    std::vector<IfaceCfg> cands;
    for (int nr : {2, 4, 8, 16}) {
        if (nr > 2 * nrhs || (nr == 16 && sizeof(R) != 4)) continue;
        for (int staged : {1, 0}) {
            IfaceCfg c;
            c.nr = nr;
            c.staged = staged;
            c.waves = 3;
            cands.push_back(c);
        }
    }
    IfaceCfg tcc;
    const bool with_tc = sizeof(R) == 4 && iface_tc_cfg(p, nrhs, tcc);
    for (const IfaceCfg& c : cands) {
        if (launch_iface<R>(ia, (int)all.subs.size(), max_rows, p->max_Lb, st, &c) != cudaSuccess) {
            (void)cudaGetLastError();
            continue;
        }
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 3; ++rep) launch_iface<R>(ia, (int)all.subs.size(), max_rows, p->max_Lb, st, &c);
        cudaEventRecord(e1, st);
        float ms = 0;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    // the tensor-core form for the stages that fill the GPU (S, on which it is timed, is
    // one of them), the best CUDA-core shape for the others
    if (with_tc && best_ms < 1e30f)
        for (int nb : {16, 32}) {
            if (nb == 32 && nrhs < 32) continue;
            const long long ctas = (long long)all.subs.size() * ((max_rows + 127) / 128) * ((nrhs + nb - 1) / nb);
            if (ctas < (tcc.tc_min_ctas >= 0 ? (long long)tcc.tc_min_ctas : 2LL * p->num_sms)) continue;
            IfaceCfg c = best;
            c.tc = tcc.tc;
            c.tc_nb = nb;
            c.tc_min_ctas = tcc.tc_min_ctas;
            if (launch_iface<R>(ia, (int)all.subs.size(), max_rows, p->max_Lb, st, &c) != cudaSuccess) {
                (void)cudaGetLastError();
                continue;
            }
            cudaEventRecord(e0, st);
            for (int rep = 0; rep < 3; ++rep) launch_iface<R>(ia, (int)all.subs.size(), max_rows, p->max_Lb, st, &c);
            cudaEventRecord(e1, st);
            float ms = 0;
            if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
                ms < best_ms) {
                best_ms = ms;
                best = c;
            }
        }
    uncount_launch(helm_launch_count() - before);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HELM_CUDA_TRY(cudaGetLastError());
    int dev_status = 0;
    HELM_CUDA_TRY(cudaMemcpyAsync(&dev_status, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CUDA_TRY(cudaStreamSynchronize(st));
    if (dev_status != 0) return take_device_status(p, "autotuning the interface stages");
    if (best_ms < 1e30f) p->iface_tuned.push_back({p->prec, nrhs, best});
    return HELM_OK;
}
static helm_status tune_shape(helm_problem* p, int nrhs, cudaStream_t st) {
    if (!p->sopts.autotune || nrhs < 2 || !p->d_K || p->prof_capture || tuned_shape(p, nrhs)) return HELM_OK;
    return p->prec == HELM_PREC_C64 ? tune_shape_t<float>(p, nrhs, st) : tune_shape_t<double>(p, nrhs, st);
}

extern "C" helm_status helm_iface_shape(const helm_problem* p, int nrhs, int* nr, int* staged, int* waves,
                                        int* tensor, int* tensor_rhs, int* tuned) {
    if (!p) return arg_error("helm_iface_shape: NULL handle");
    IfaceCfg tmp;
    const IfaceCfg* c = iface_shape_for(p, nrhs, tmp);
    IfaceCfg d;
    d.nr = nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1;
    if (!c) c = &d;
    if (nr) *nr = c->nr;
    if (staged) *staged = c->staged;
    if (waves) *waves = c->waves;
    if (tensor) *tensor = c->tc;
    if (tensor_rhs) *tensor_rhs = c->tc ? c->tc_nb : 0;
    if (tuned) *tuned = tuned_shape(p, nrhs) != nullptr;
    return HELM_OK;
}

// autotuned launch shape of the full stages for nrhs RHS (nullptr: the kernels' rules)
static const StageCfg* stage_shape_for(const helm_problem* p, int nrhs) {
    for (const auto& t : p->stage_tuned)
        if (t.prec == p->prec && t.nrhs == nrhs) return &t.cfg;
    return nullptr;
}

template <typename R>
static helm_status run_stage_t(helm_problem* p, const PcWork& w, const PcCtx& cx, const StageDesc& sd,
                               const double2* r, double2* z, int nrhs, cudaStream_t st);

// The autotuner of the full-stage kernels (the liftings and reconstructions, which
// stream the factors): the first application with a given RHS count times the lifting
// stage (every subdomain; it reads r and writes B and X, so it may run any number of
// times) for each candidate shape with CUDA events on the caller's stream, and keeps
// the fastest: on the CUDA cores, one or two CTAs per subdomain (the second taking one
// column half of the factors, halves of the next input exchanged through distributed
// shared memory) and the factor chunk per ring slot (64, 48, 32 KB); in the tensor-core
// form, 16, 32 or 64 RHS per CTA.  Not while a stream is being captured.
template <typename R>
static helm_status tune_stage_t(helm_problem* p, const double2* r, int nrhs, cudaStream_t st) {
    const PcWork w{{p->d_trace[0], p->d_trace[1], p->d_trace[2], p->d_trace[3]}, p->d_yws, p->d_pc_norm,
                   p->d_pc_partial, p->d_escr, p->d_r64};
    const PcCtx cx = precond_prologue<R>(p, w, r, nrhs, st);
    StageDesc lift = p->sched[HELM_SCHED_BSP].front();
    lift.final_ = 0;
    if (lift.mask == 0) lift.dst = lift.dst2 = BUF_NONE;     // one subdomain: no traces
    std::vector<StageCfg> cands;
    if (cx.tc) {
        for (int nr : {16, 32, 64}) {
            if (nr > nrhs && nr > 16) continue;
            if (nr == 64 && (p->tc_split != 1 || p->tc_mt != 1)) continue;
            if (nr == 32 && p->tc_split == 3 && p->tc_mt != 1) continue;
            StageCfg c;
            c.tc_nr = nr;
            cands.push_back(c);
        }
    } else {
        for (int cs : {1, 2})
            for (int kb : {64, 48, 32}) {
                StageCfg c;
                c.csize = cs;
                c.chunk_kb = kb;
                cands.push_back(c);
            }
    }
    if (cands.size() < 2) return HELM_OK;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    HELM_CUDA_TRY(cudaEventCreate(&e0));
    HELM_CUDA_TRY(cudaEventCreate(&e1));
    const long long before = helm_launch_count();
    const int prof_was = p->prof_on;
    p->prof_on = 0;
    StageCfg best{};
    float best_ms = 1e30f;
    for (const StageCfg& c : cands) {
        p->stage_try = &c;
        if (run_stage_t<R>(p, w, cx, lift, r, nullptr, nrhs, st) != HELM_OK) {   // warm (and validity)
            (void)cudaGetLastError();
            continue;
        }
        cudaEventRecord(e0, st);
        for (int rep = 0; rep < 3; ++rep) run_stage_t<R>(p, w, cx, lift, r, nullptr, nrhs, st);
        cudaEventRecord(e1, st);
        float ms = 0;
        if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess &&
            ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    p->stage_try = nullptr;
    p->prof_on = prof_was;
    uncount_launch(helm_launch_count() - before);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    HELM_CUDA_TRY(cudaGetLastError());
    int dev_status = 0;
    HELM_CUDA_TRY(cudaMemcpyAsync(&dev_status, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
    HELM_CUDA_TRY(cudaStreamSynchronize(st));
    if (dev_status != 0) return take_device_status(p, "autotuning the stage kernels");
    if (best_ms < 1e30f) p->stage_tuned.push_back({p->prec, nrhs, best});
    return HELM_OK;
}
static helm_status tune_stage(helm_problem* p, const double2* r, int nrhs, cudaStream_t st) {
    if (!p->sopts.autotune || p->prof_capture || stage_shape_for(p, nrhs)) return HELM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return HELM_OK;
    return p->prec == HELM_PREC_C64 ? tune_stage_t<float>(p, r, nrhs, st) : tune_stage_t<double>(p, r, nrhs, st);
}

extern "C" helm_status helm_stage_shape(const helm_problem* p, int nrhs, int* csize, int* chunk_kb, int* tensor_rhs,
                                        int* tuned) {
    if (!p) return arg_error("helm_stage_shape: NULL handle");
    const StageCfg* c = stage_shape_for(p, nrhs);
    const StageCfg d{};
    if (!c) c = &d;
    if (csize) *csize = c->csize;
    if (chunk_kb) *chunk_kb = c->chunk_kb;
    if (tensor_rhs) *tensor_rhs = c->tc_nr;
    if (tuned) *tuned = c != &d;
    return HELM_OK;
}

template <typename R>
static helm_status run_stage_t(helm_problem* p, const PcWork& w, const PcCtx& cx, const StageDesc& sd,
                               const double2* r, double2* z, int nrhs, cudaStream_t st) {
    using T = Cx<R>;
    const double* rinv = cx.rinv;
    const double* rsc = cx.rsc;
    const bool tc = cx.tc;
    T* buf[4] = {(T*)w.trace[0], (T*)w.trace[1], (T*)w.trace[2], (T*)w.trace[3]};
    auto B = [&](int id) -> T* { return id < 0 ? nullptr : buf[id]; };
    NvtxRange nvtx(sd.iface ? "interface stage" : sd.final_ ? "reconstruction stage" : sd.src ? "lifting stage"
                                                                                              : "full stage");
    if (sd.iface && p->d_K) {
        IfaceArgs<R> ia{};
        ia.subtab = p->d_subtab;
        ia.subs = p->d_stage_subs + sd.sub_off;
        ia.nrhs = nrhs;
        ia.ntrace = p->ntrace;
        ia.K = (const T*)stage_kmat(p, sd.kmat);
        ia.tc = stage_tc<T>(p);
        ia.gin0 = B(sd.in0); ia.gin1 = B(sd.in1);
        ia.mask = sd.mask;
        ia.dst = B(sd.dst); ia.dst2 = B(sd.dst2); ia.base = B(sd.base); ia.sub = B(sd.sub);
        ia.err = p->d_err;
        ia.part = p->d_tcpart; ia.part_cap = p->tcpart_cap;
        ia.cnt = p->d_tccnt; ia.cnt_cap = p->tccnt_cap;
        // grid rows: the most output rows (points of the masked sides) of a subdomain
        int max_rows = 0;
        for (int id : sd.subs) {
            const SubDev& d = p->subs[id].dev;
            int rows = 0;
            for (int sde = 0; sde < 4; ++sde)
                if ((sd.mask & (1 << sde)) && d.bo[sde] >= 0) rows += (sde == SW || sde == SE) ? d.my : d.mx;
            max_rows = std::max(max_rows, rows);
        }
        // one complex64 RHS applying K itself: the packed symmetric tiles
        const bool sym = sizeof(R) == 4 && nrhs == 1 && p->d_Kp && sd.kmat == KMAT_K && sd.mask == 15 &&
                         sd.subs.size() == p->subs.size();
        double bytes = 0, flops = 0;
        if (p->prof_on) iface_accounting(p, sd, nrhs, sizeof(T), bytes, flops, sym);
        prof_begin(p, HELM_K_TRACE, st);
        IfaceCfg tmp;
        cudaError_t e;
        if constexpr (sizeof(R) == 4) {
            if (sym) {
                ia.Kp = p->d_Kp;
                e = launch_iface_sym(ia, p->d_symrt, p->sym_nrt, p->max_Lb, p->num_sms, st);
            } else {
                e = launch_iface<R>(ia, (int)sd.subs.size(), max_rows, p->max_Lb, st, iface_shape_for(p, nrhs, tmp));
            }
        } else {
            e = launch_iface<R>(ia, (int)sd.subs.size(), max_rows, p->max_Lb, st, iface_shape_for(p, nrhs, tmp));
        }
        prof_end(p, HELM_K_TRACE, bytes, st, flops);
        if (e != cudaSuccess) return cuda_status(e, "interface stage launch");
        return HELM_OK;
    }
    StageArgs<R> a{};
    a.subtab = p->d_subtab;
    a.subs = p->d_stage_subs + sd.sub_off;
    a.nx = p->nx; a.ny = p->ny; a.nrhs = nrhs;
    a.ntrace = p->ntrace;
    a.wstride = p->N();
    a.X = (const T*)p->d_X;
    a.tc = stage_tc<T>(p);
    a.src = sd.src;
    a.r = r;
    a.rscale = rinv;
    a.gin0 = B(sd.in0); a.gin1 = B(sd.in1);
    a.mask = sd.mask;
    a.dst = B(sd.dst); a.dst2 = B(sd.dst2); a.base = B(sd.base); a.sub = B(sd.sub);
    a.z = sd.final_ ? z : nullptr;
    a.zscale = rsc;
    a.yws = (T*)w.yws;
    a.err = p->d_err;
    double bytes = 0, flops = 0;
    if (p->prof_on) {
        // algorithmic bytes: each X_r once per stage (shared by all RHS), the
        // solve workspace y written and read once, source read, volume output
        // written, incoming traces read, outgoing traces (and their base/sub) moved
        const double sT = sizeof(T);
        for (int id : sd.subs) {
            const SubDev& d = p->subs[id].dev;
            double per_rhs = 2.0 * (d.my - 1) * d.mx * sT;
            if (sd.src) per_rhs += 16.0 * d.mx * d.my;
            if (sd.final_) per_rhs += 16.0 * d.mx * d.my;
            for (int sde = 0; sde < 4; ++sde) {
                if (d.tin[sde] < 0) continue;
                const double len = (sde == SW || sde == SE) ? d.my : d.mx;
                if (sd.in0 >= 0) per_rhs += len * sT;
                if (sd.in1 >= 0) per_rhs += len * sT;
                if (sd.mask & (1 << sde))
                    per_rhs += len * sT * (1 + (sd.dst2 >= 0) + (sd.base >= 0) + (sd.sub >= 0));
            }
            bytes += (2.0 * d.my - 1) * d.mx * (double)d.mx * sT + per_rhs * nrhs;
            flops += 8.0 * (2.0 * d.my - 1) * d.mx * (double)d.mx * nrhs;
        }
    }
    const StageCfg* scfg = p->stage_try ? p->stage_try : stage_shape_for(p, nrhs);
    prof_begin(p, HELM_K_STAGE, st);
    cudaError_t e = cudaSuccess;
    bool done = false;
    if constexpr (sizeof(R) == 4) {
        // 16 or more right-hand sides: the block solves are GEMMs for the tensor cores
        if (tc) {
            for (int c = 0; c < 2 && e == cudaSuccess; ++c) {
                StageArgs<R> ac = a;
                ac.escr = (T*)w.escr;
                ac.uscr = (T*)w.escr + (long long)nrhs * p->etot;
                ac.estride = p->etot;
                ac.r64 = (const T*)w.r64;
                ac.subs = p->d_stage_subs + sd.tc_off[c];
                e = launch_tc_stage(ac, p->d_XT, c + 1, p->tc_split, sd.tc_n[c], st, scfg ? scfg->tc_nr : 0);
            }
            done = true;
        }
    }
    if (!done)
        e = launch_stage<R>(a, (int)sd.subs.size(), p->max_mx, p->max_my, p->max_w, p->max_ld, p->num_sms, st, scfg);
    prof_end(p, HELM_K_STAGE, bytes, st, flops);
    if (e != cudaSuccess) return cuda_status(e, "stage launch");
    return HELM_OK;
}

// With the HABC transmission the lifting is a base solve of the source whose boundary
// values u_f (written as outgoing data with the identity coefficients, i.e. into the
// neighbours' slots) are swapped into U, then b = Lq u_f as an interface stage into
// the lifting's outputs (k_habc.cu)
template <typename R>
static helm_status habc_lifting_t(helm_problem* p, const PcWork& w, const PcCtx& cx, const StageDesc& lift,
                                  const double2* r, int nrhs, cudaStream_t st) {
    using T = Cx<R>;
    StageDesc a = lift;
    a.dst = BUF_B; a.dst2 = BUF_NONE; a.base = a.sub = BUF_NONE; a.mask = 15; a.final_ = 0;
    helm_status s = run_stage_t<R>(p, w, cx, a, r, nullptr, nrhs, st);
    if (s != HELM_OK) return s;
    launch_trace_swap<T>((const T*)w.trace[BUF_B], (T*)w.trace[BUF_U], p->d_swap, p->ntrace, nrhs, st);
    StageDesc g = lift;
    g.iface = 1; g.src = 0; g.in0 = BUF_U; g.in1 = BUF_NONE; g.mask = 15; g.final_ = 0; g.kmat = KMAT_LQ;
    return run_stage_t<R>(p, w, cx, g, r, nullptr, nrhs, st);
}
// ... and the reconstruction a base solve with the source and the boundary datum
// D1 g + D2 u_f (g = in0 (+ in1)): D2 u_f into t1, D1 g + t1 into t2 (both in the
// neighbours' slots), swapped into t1, the incoming data of the base solves
template <typename R>
static helm_status habc_recon_t(helm_problem* p, const PcWork& w, const PcCtx& cx, const StageDesc& rec, int in0,
                                int in1, int t1, int t2, const double2* r, double2* z, int nrhs, cudaStream_t st) {
    using T = Cx<R>;
    StageDesc g = rec;
    g.iface = 1; g.src = 0; g.mask = 15; g.dst2 = BUF_NONE; g.sub = BUF_NONE; g.final_ = 0;
    g.in0 = BUF_U; g.in1 = BUF_NONE; g.base = BUF_NONE; g.dst = t1; g.kmat = KMAT_D2;
    helm_status s = run_stage_t<R>(p, w, cx, g, r, nullptr, nrhs, st);
    if (s != HELM_OK) return s;
    g.in0 = in0; g.in1 = in1; g.base = t1; g.dst = t2; g.kmat = KMAT_D1;
    s = run_stage_t<R>(p, w, cx, g, r, nullptr, nrhs, st);
    if (s != HELM_OK) return s;
    launch_trace_swap<T>((const T*)w.trace[t2], (T*)w.trace[t1], p->d_swap, p->ntrace, nrhs, st);
    StageDesc f = rec;
    f.in0 = t1; f.in1 = BUF_NONE;
    return run_stage_t<R>(p, w, cx, f, r, z, nrhs, st);
}

template <typename R>
static helm_status run_precond_t(helm_problem* p, const PcWork& w, int sched, const double2* r, double2* z, int nrhs,
                                 cudaStream_t st) {
    const PcCtx cx = precond_prologue<R>(p, w, r, nrhs, st);
    const std::vector<StageDesc>& stg = p->sched[sched];
    const bool habc = p->habc && stg.size() > 2;
    for (size_t i = 0; i < stg.size(); ++i) {
        if (habc && i == 0) {
            const helm_status s = habc_lifting_t<R>(p, w, cx, stg[0], r, nrhs, st);
            if (s != HELM_OK) return s;
            continue;
        }
        if (habc && i + 1 == stg.size()) {
            // after the sweep B is free (and U once D2 has read it)
            return habc_recon_t<R>(p, w, cx, stg[i], stg[i].in0, stg[i].in1, BUF_B, BUF_U, r, z, nrhs, st);
        }
        if (i == 1 && stg.size() > 2) {
            helm_status s = HELM_OK;
            if (run_sweep_persistent<R>(p, w, sched, nrhs, st, s)) {
                if (s != HELM_OK) return s;
                i = stg.size() - 2;                  // continue with the reconstruction
                continue;
            }
        }
        const helm_status s = run_stage_t<R>(p, w, cx, stg[i], r, z, nrhs, st);
        if (s != HELM_OK) return s;
    }
    return HELM_OK;
}

static helm_status run_precond(helm_problem* p, int sched, const double2* r, double2* z, int nrhs, cudaStream_t st) {
    helm_status s = ensure_pc_ws(p, nrhs);
    if (s != HELM_OK) return s;
    s = tune_shape(p, nrhs, st);
    if (s != HELM_OK) return s;
    s = tune_stage(p, r, nrhs, st);
    if (s != HELM_OK) return s;
    const PcWork w{{p->d_trace[0], p->d_trace[1], p->d_trace[2], p->d_trace[3]}, p->d_yws, p->d_pc_norm,
                   p->d_pc_partial, p->d_escr, p->d_r64};
    return p->prec == HELM_PREC_C64 ? run_precond_t<float>(p, w, sched, r, z, nrhs, st)
                                    : run_precond_t<double>(p, w, sched, r, z, nrhs, st);
}

// The same application replayed from a captured CUDA graph: the first call for a
// (schedule, nrhs, r, z) captures the launch sequence on an internal stream (the
// caller's stream may be the legacy default stream, which cannot be captured);
// every call launches the executable graph on the caller's stream.
static helm_status run_precond_graph(helm_problem* p, int sched, const double2* r, double2* z, int nrhs,
                                     cudaStream_t st) {
    if (p->prof_on) return run_precond(p, sched, r, z, nrhs, st);   // per-launch events need plain launches
    helm_status s = ensure_pc_ws(p, nrhs);
    if (s != HELM_OK) return s;
    s = tune_shape(p, nrhs, st);
    if (s != HELM_OK) return s;
    s = tune_stage(p, r, nrhs, st);
    if (s != HELM_OK) return s;
    for (const auto& g : p->graphs)
        if (g.sched == sched && g.nrhs == nrhs && g.r == r && g.z == z) {
            HELM_CUDA_TRY(cudaGraphLaunch(g.exec, st));
            count_launch((int)g.kernels);
            return HELM_OK;
        }
    if (p->graphs.size() >= 1024) drop_graphs(p);
    if (!p->cap_stream) {
        HELM_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        HELM_CUDA_TRY(cudaEventCreateWithFlags(&p->cap_ev, cudaEventDisableTiming));
    }
    const long long before = helm_launch_count();
    HELM_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
    s = run_precond(p, sched, r, z, nrhs, p->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->cap_stream, &graph);
    const long long kernels = helm_launch_count() - before;
    uncount_launch(kernels);                                          // captured, not launched
    if (s != HELM_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (ec != cudaSuccess) return cuda_status(ec, "capturing the preconditioner");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_status(ei, "instantiating the preconditioner graph");
    p->graphs.push_back({sched, nrhs, r, z, exec, kernels});
    HELM_CUDA_TRY(cudaGraphLaunch(exec, st));
    count_launch((int)kernels);
    return HELM_OK;
}

// A launch sequence with fixed pointers replayed from a CUDA graph: captured on
// the first call for (tag, nrhs) on the internal stream, launched on `st`.
// Plain launches while profiling (the per-launch events need them).
static helm_status run_captured(helm_problem* p, int tag, int nrhs, cudaStream_t st,
                                const std::function<helm_status(cudaStream_t)>& seq) {
    const void* key = reinterpret_cast<const void*>((intptr_t)(tag + 1));
    auto replay = [&](const helm_problem::PcGraph& g) -> helm_status {
        // while profiling, one event pair brackets the whole sequence of its class
        if (g.cls >= 0) prof_begin(p, g.cls, st);
        HELM_CUDA_TRY(cudaGraphLaunch(g.exec, st));
        if (g.cls >= 0 && p->prof_on) {
            prof_end(p, g.cls, g.cls_bytes, st, g.cls_flops);
            p->prof[g.cls].kernels += g.cls_kernels - 1;
        }
        count_launch((int)g.kernels);
        return HELM_OK;
    };
    for (const auto& g : p->graphs)
        if (g.sched == -1 && g.nrhs == nrhs && g.r == key) return replay(g);
    if (!p->cap_stream) {
        HELM_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
        HELM_CUDA_TRY(cudaEventCreateWithFlags(&p->cap_ev, cudaEventDisableTiming));
    }
    const long long before = helm_launch_count();
    // capture with the per-class accounting switched on (no events are recorded)
    const int prof_was = p->prof_on;
    p->prof_on = 1;
    p->prof_capture = 1;
    for (int k = 0; k < 5; ++k) { p->cap_bytes[k] = p->cap_flops[k] = 0; p->cap_kernels[k] = 0; }
    HELM_CUDA_TRY(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
    helm_status s = seq(p->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(p->cap_stream, &graph);
    p->prof_capture = 0;
    p->prof_on = prof_was;
    const long long kernels = helm_launch_count() - before;
    uncount_launch(kernels);
    if (s != HELM_OK) { if (graph) cudaGraphDestroy(graph); return s; }
    if (ec != cudaSuccess) return cuda_status(ec, "capturing a stage sequence");
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_status(ei, "instantiating a stage-sequence graph");
    helm_problem::PcGraph g{-1, nrhs, key, nullptr, exec, kernels};
    for (int k = 0; k < 5; ++k)
        if (p->cap_kernels[k] > 0 && (g.cls < 0 || p->cap_kernels[k] > g.cls_kernels)) { g.cls = k; g.cls_kernels = p->cap_kernels[k]; }
    for (int k = 0; k < 5; ++k) { g.cls_bytes += p->cap_bytes[k]; g.cls_flops += p->cap_flops[k]; }
    p->graphs.push_back(g);
    return replay(p->graphs.back());
}

extern "C" helm_status precond_apply(helm_problem* p, int sched, const helm_c128* r, helm_c128* z, int nrhs,
                                     void* stream) {
    NvtxRange nvtx("precond_apply");
    if (!p) return arg_error("precond_apply: NULL handle");
    if (!p->factored) { set_error("precond_apply: call precond_factor first"); return HELM_ERR_STATE; }
    if ((sched < 0 || sched >= HELM_NSCHED)) return arg_error("precond_apply: unknown schedule");
    if (nrhs < 0) return arg_error("precond_apply: nrhs < 0");
    if (nrhs == 0) return HELM_OK;
    if (!r || !z) return arg_error("precond_apply: NULL array");
    const size_t vb = (size_t)p->N() * nrhs * sizeof(double2);
    HcCall hcc{{r, vb}, {z, vb}};
    return run_precond(p, sched, (const double2*)r, (double2*)z, nrhs, (cudaStream_t)stream);
}

// ---------------------------------------------- preconditioner without allocation
// Scratch of precond_apply_noalloc: one fixed array in device memory, part of the
// library image, so every GPU that loads the library holds these bytes until the
// process exits.  All calls share it (see include/helm.h).
static __device__ __align__(256) unsigned char g_noalloc_scratch[HELM_NOALLOC_SCRATCH_BYTES];

// device address of g_noalloc_scratch per device ordinal, looked up on the first
// call made with that device current (host code cannot use the symbol itself)
static std::atomic<void*> g_noalloc_ptr[128];

extern "C" helm_status precond_apply_noalloc(helm_problem* p, int sched, const helm_c128* r, helm_c128* z, int nrhs,
                                             void* stream) {
    NvtxRange nvtx("precond_apply_noalloc");
    if (!p) return arg_error("precond_apply_noalloc: NULL handle");
    if (!p->factored) { set_error("precond_apply_noalloc: call precond_factor first"); return HELM_ERR_STATE; }
    if ((sched < 0 || sched >= HELM_NSCHED)) return arg_error("precond_apply_noalloc: unknown schedule");
    if (nrhs < 0) return arg_error("precond_apply_noalloc: nrhs < 0");
    if (nrhs == 0) return HELM_OK;
    if (!r || !z) return arg_error("precond_apply_noalloc: NULL array");
    // carve the scratch: 3 interface buffers, the solve workspace, norms, partial sums
    const size_t elem = p->prec == HELM_PREC_C64 ? sizeof(float2) : sizeof(double2);
    auto round256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t tbytes = round256((size_t)p->ntrace * nrhs * elem);
    const size_t ybytes = round256((size_t)p->N() * nrhs * elem);
    const size_t nbytes = round256((size_t)3 * nrhs * sizeof(double));
    const size_t pbytes = round256((size_t)kPartialBlocks * nrhs * sizeof(double));
    const bool tc = p->prec == HELM_PREC_C64 && tc_used(p, nrhs);
    const size_t ebytes = tc ? round256((size_t)2 * p->etot * nrhs * sizeof(float2)) : 0;
    const size_t rbytes = tc ? round256((size_t)p->N() * nrhs * sizeof(float2)) : 0;
    const int nbuf = p->habc ? 4 : 3;                 // the HABC keeps the liftings' boundary values
    const size_t need = nbuf * tbytes + ybytes + nbytes + pbytes + ebytes + rbytes;
    if (need > (size_t)HELM_NOALLOC_SCRATCH_BYTES) {
        char buf[256];
        snprintf(buf, sizeof buf,
                 "precond_apply_noalloc: needs %zu bytes of scratch for %d right-hand sides, more than the fixed "
                 "%d bytes; use precond_apply or fewer right-hand sides per call",
                 need, nrhs, (int)HELM_NOALLOC_SCRATCH_BYTES);
        set_error(buf);
        return HELM_ERR_ARG;
    }
    int dev = 0;
    HELM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return arg_error("precond_apply_noalloc: device ordinal out of range");
    void* base = g_noalloc_ptr[dev].load();
    if (!base) {
        cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
        if (e != cudaSuccess || !base) return cuda_status(e, "precond_apply_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev].store(base);
    }
    const size_t vb = (size_t)p->N() * nrhs * sizeof(double2);
    HcCall hcc{{r, vb}, {z, vb}, {base, (size_t)HELM_NOALLOC_SCRATCH_BYTES}};
    unsigned char* b = (unsigned char*)base;
    unsigned char* v = b + nbuf * tbytes;             // after the interface buffers
    unsigned char* tail = v + ybytes + nbytes + pbytes;
    PcWork w{{b, b + tbytes, b + 2 * tbytes, nbuf == 4 ? b + 3 * tbytes : nullptr}, v, (double*)(v + ybytes),
             (double*)(v + ybytes + nbytes), tc ? tail : nullptr, tc ? tail + ebytes : nullptr};
    cudaStream_t st = (cudaStream_t)stream;
    return p->prec == HELM_PREC_C64 ? run_precond_t<float>(p, w, sched, (const double2*)r, (double2*)z, nrhs, st)
                                    : run_precond_t<double>(p, w, sched, (const double2*)r, (double2*)z, nrhs, st);
}

extern "C" helm_status helm_matvec(helm_problem* p, const helm_c128* u, helm_c128* Au, int nrhs, void* stream) {
    NvtxRange nvtx("helm_matvec");
    if (!p) return arg_error("helm_matvec: NULL handle");
    if (nrhs < 0) return arg_error("helm_matvec: nrhs < 0");
    if (nrhs == 0) return HELM_OK;
    if (!u || !Au) return arg_error("helm_matvec: NULL array");
    const size_t vb = (size_t)p->N() * nrhs * sizeof(double2);
    HcCall hcc{{u, vb}, {Au, vb}};
    launch_matvec(p->d_adiag, p->nx, p->ny, (const double2*)u, (double2*)Au, nrhs, (cudaStream_t)stream);
    HELM_CUDA_TRY(cudaGetLastError());
    return HELM_OK;
}

// ------------------------------------------------------------------ FGMRES
// with_bx: also the right-hand side and solution arrays of the interface solver
static helm_status ensure_kw(KrylovWS& w, int nrhs, int m, long long n, bool with_bx) {
    if (w.nrhs >= nrhs && w.restart >= m && w.n == n && (!with_bx || w.b)) return HELM_OK;
    free_kw(w);
    const int nb = kPartialBlocks;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
    chk(dalloc(w.V, (size_t)(m + 1) * nrhs * n));
    chk(dalloc(w.Z, (size_t)m * nrhs * n));
    chk(dalloc(w.H, (size_t)nrhs * (m + 1) * m));
    chk(dalloc(w.cs, (size_t)nrhs * (m + 1)));
    chk(dalloc(w.sn, (size_t)nrhs * (m + 1)));
    chk(dalloc(w.g, (size_t)nrhs * (m + 1)));
    chk(dalloc(w.h1, (size_t)nrhs * (m + 1)));
    chk(dalloc(w.h2, (size_t)nrhs * (m + 1)));
    chk(dalloc(w.hsum, (size_t)nrhs * (m + 1)));
    chk(dalloc(w.y, (size_t)nrhs * (m + 1)));
    chk(dalloc(w.cpart, (size_t)nb * nrhs * (m + 1)));
    chk(dalloc(w.rpart, (size_t)nb * nrhs));
    chk(dalloc(w.rn, (size_t)4 * nrhs));
    chk(dalloc(w.need, (size_t)nrhs));
    {
        const int g = mgs_grid();
        if (g > 0) {
            // two halves of per-CTA partials: one value (modified Gram-Schmidt) or j + 2
            // values per RHS of a group (the fused classical step) per CTA
            chk(dalloc(w.mgs_part, (size_t)2 * g * (m + 2) * 16));   // groups of up to 16 RHS (k_mgs.cu)
            chk(dalloc(w.mgs_bar, (size_t)2));
            if (e == cudaSuccess) e = cudaMemset(w.mgs_bar, 0, 2 * sizeof(unsigned));
        }
    }
    chk(dalloc(w.est, (size_t)nrhs));
    chk(dalloc(w.invh, (size_t)nrhs));
    chk(dalloc(w.ctl, (size_t)4));
    chk(dalloc(w.iters, (size_t)nrhs));
    chk(dalloc(w.thr, (size_t)nrhs));
    chk(dalloc(w.active, (size_t)nrhs));
    chk(dalloc(w.jcount, (size_t)nrhs));
    if (with_bx) {
        chk(dalloc(w.b, (size_t)nrhs * n));
        chk(dalloc(w.x, (size_t)nrhs * n));
    }
    if (e != cudaSuccess) { free_kw(w); return cuda_status(e, "allocating the Krylov workspace"); }
    static long long kw_generation = 0;
    w.gen = ++kw_generation;
    w.nrhs = nrhs;
    w.restart = m;
    w.n = n;
    // partial-sum blocks of the reductions: ~128 elements per block for short
    // (interface) vectors, at least one per SM, at most the allocated count
    w.nblk = (int)std::min<long long>(nb, std::max<long long>(152, (n + 127) / 128));
    return HELM_OK;
}

__global__ void add_cols_kernel(const double2* a, const double2* b, double2* c, int n, int nrhs, int ld) {
    int k = blockIdx.x, i = threadIdx.x;
    for (; i < n; i += blockDim.x) {
        double2 x = a[k * ld + i], y = b[k * ld + i];
        c[k * ld + i] = make_double2(x.x + y.x, x.y + y.y);
    }
}

// Selective reorthogonalisation (Daniel-Gragg-Kaufman-Stewart): after one
// classical Gram-Schmidt pass w' = w - V h1, a second pass is needed only when
// the projection cancelled most of w, ||w'||^2 < eta2 ||w||^2 (eta2 = 1/2: ||w'|| < ||w|| / sqrt(2)).
// n2[k] = ||w||^2 (before), n2[nrhs + k] = ||w'||^2 (after the first pass).
__global__ void dgks_decide_kernel(const double* n2, const int* active, int* need, int nrhs, double eta2) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    need[k] = (active[k] && n2[nrhs + k] < eta2 * n2[k]) ? 1 : 0;
}
// hnorm[k] = sqrt(need ? ||w''||^2 : ||w'||^2)
__global__ void dgks_norm_kernel(const double* n2, const int* need, double* hnorm, int nrhs) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nrhs) return;
    hnorm[k] = sqrt(need[k] ? n2[2 * nrhs + k] : n2[nrhs + k]);
}

// The operator, preconditioner and residual of one FGMRES: vectors of n values
// per RHS, RHS k at offset k*n, of type VT (double2, or float2 for the interface
// iterations with complex64 factors).
template <typename VT>
struct KrylovOps {
    std::function<helm_status(const VT* x, bool x_zero, VT* r)> residual;   // r = b - A x
    std::function<helm_status(const VT* v, VT* z)> precond;                // z = M^{-1} v
    std::function<helm_status(const VT* z, VT* w)> matvec;                 // w = A z
    // optional, for the device-driven loop: enqueue precond + matvec of Arnoldi step j = *dj
    // (z_j = M^{-1} v_j into Z, w = A z_j into V slot j + 1) on stream cs without host work
    // that depends on j, so that one capture serves every step
    std::function<helm_status(cudaStream_t cs, VT* V, VT* Z, long long vsk, const int* dj)> dev_step;
    // optional refinements of dev_step: the operator's output is left negated in dev_w_src
    // (instead of in V slot j + 1) for the Gram-Schmidt step to read, which also writes
    // v_{j+1} into dev_v_out1/2 (the next step's input); dev_prologue(cs, V) prepares
    // the first step's input from V slot 0
    VT* dev_w_src = nullptr;
    VT* dev_v_out1 = nullptr;
    VT* dev_v_out2 = nullptr;
    std::function<helm_status(cudaStream_t cs, VT* V)> dev_prologue;
    int dev_tag = 0;   // identifies what dev_step enqueues (schedule, form): part of the graph key
    // selective reorthogonalisation: a second Gram-Schmidt pass when ||w'||^2 < reorth ||w||^2
    double reorth = 0.5;
};

// One restart cycle of FGMRES with the Arnoldi steps driven on the device (see
// fgmres_core): the step (ops.dev_step, the fused Gram-Schmidt step and the loop
// control, j read from kw.ctl) is captured once per workspace into the body of a
// conditional while node; each cycle uploads the counters, launches the graph and
// reads back the steps taken.  cycle_done = true when the cycle ran here; false
// (and the host-driven loop runs instead) when the graph could not be built.
template <typename VT>
static helm_status device_cycle(helm_problem* p, KrylovWS& kw, long long N, int nrhs, int m, int maxit, double tol,
                                const std::vector<double>& bnorm, const KrylovOps<VT>& ops, int grid,
                                std::vector<int>& iters, std::vector<int>& active, std::vector<int>& jcount,
                                bool& cycle_done, const char* who, cudaStream_t st) {
    cycle_done = false;
    const long long vsk = (long long)nrhs * N;
    const int ld = m + 1;
    VT* const KV = reinterpret_cast<VT*>(kw.V);
    VT* const KZ = reinterpret_cast<VT*>(kw.Z);
    const void* key = reinterpret_cast<const void*>((intptr_t)(1000 + (int)sizeof(VT) + 64 * ops.dev_tag));
    helm_problem::PcGraph* gr = nullptr;
    for (auto& g : p->graphs)
        if (g.sched == -2 && g.r == key && g.nrhs == nrhs && g.gen == kw.gen && g.m == m && g.limit == p->wait_cycles)
            gr = &g;
    if (!gr) {
        // graphs of earlier workspaces hold freed pointers: drop them
        for (size_t i = 0; i < p->graphs.size();) {
            auto& g = p->graphs[i];
            if (g.sched == -2 && g.r == key) {
                cudaGraphExecDestroy(g.exec);
                if (g.tmpl) cudaGraphDestroy(g.tmpl);
                p->graphs.erase(p->graphs.begin() + (long)i);
            } else {
                ++i;
            }
        }
        if (!p->cap_stream) {
            HELM_CUDA_TRY(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking));
            HELM_CUDA_TRY(cudaEventCreateWithFlags(&p->cap_ev, cudaEventDisableTiming));
        }
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        bool ok = cudaGraphCreate(&graph, 0) == cudaSuccess;
        cudaGraphConditionalHandle h{};
        cudaGraph_t body = nullptr;
        if (ok) ok = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        if (ok) {
            cudaGraphNodeParams np = {};
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            cudaGraphNode_t node;
            ok = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) == cudaSuccess;
            if (ok) body = np.conditional.phGraph_out[0];
        }
        long long step_kernels = 0;
        if (ok) ok = cudaStreamBeginCaptureToGraph(p->cap_stream, body, nullptr, nullptr, 0,
                                                   cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
            const long long before = helm_launch_count();
            helm_status q = ops.dev_step(p->cap_stream, KV, KZ, vsk, kw.ctl);
            cudaError_t e = cudaSuccess;
            if (q == HELM_OK)
                e = launch_cgs2_step<VT>(KV, vsk, N, 0, N, nrhs, kw.active, kw.hsum, ld, kw.rn + 3 * nrhs, kw.need,
                                         kw.H, ld, (long long)ld * m, kw.cs, kw.sn, kw.g, ld, kw.est, kw.invh,
                                         kw.mgs_part, kw.mgs_bar, p->d_err, grid, p->cap_stream, kw.ctl, m - 1,
                                         ops.dev_w_src, ops.dev_v_out1, ops.dev_v_out2, p->wait_cycles, ops.reorth);
            if (q == HELM_OK && e == cudaSuccess)
                launch_arnoldi_ctl(kw.ctl, kw.est, kw.thr, kw.active, kw.iters, kw.jcount, maxit, nrhs, p->d_err, h,
                                   p->cap_stream);
            cudaGraph_t out = nullptr;
            const cudaError_t ec = cudaStreamEndCapture(p->cap_stream, &out);
            step_kernels = helm_launch_count() - before;
            uncount_launch(step_kernels);
            ok = q == HELM_OK && e == cudaSuccess && ec == cudaSuccess;
            if (q != HELM_OK) { cudaGraphDestroy(graph); return q; }
        }
        if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
        if (!ok) {
            // conditional graphs unavailable here: the host-driven loop from now on
            (void)cudaGetLastError();
            if (graph) cudaGraphDestroy(graph);
            p->dev_loop_broken = true;
            return HELM_OK;
        }
        helm_problem::PcGraph g{-2, nrhs, key, nullptr, exec, step_kernels};
        g.tmpl = graph;
        g.gen = kw.gen;
        g.m = m;
        g.limit = p->wait_cycles;
        p->graphs.push_back(g);
        gr = &p->graphs.back();
    }
    // counters of this cycle: j = 0, the restart length, maxit; the steps taken so far
    // and the stopping thresholds per RHS (active is already on the device)
    {
        const int ctl[4] = {0, m, maxit, 0};
        std::vector<double> thr(nrhs);
        for (int k = 0; k < nrhs; ++k) thr[k] = tol * bnorm[k];
        HELM_CUDA_TRY(cudaMemcpyAsync(kw.ctl, ctl, sizeof(ctl), cudaMemcpyHostToDevice, st));
        HELM_CUDA_TRY(cudaMemcpyAsync(kw.iters, iters.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        HELM_CUDA_TRY(cudaMemcpyAsync(kw.thr, thr.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
        // zero for every RHS (the steps of the active ones are counted on the device)
        HELM_CUDA_TRY(cudaMemcpyAsync(kw.jcount, jcount.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        if (ops.dev_prologue) {
            helm_status q = ops.dev_prologue(st, KV);
            if (q != HELM_OK) return q;
        }
        HELM_CUDA_TRY(cudaGraphLaunch(gr->exec, st));
        int ctl_out[4] = {0, 0, 0, 0};
        int dev_status = 0;
        HELM_CUDA_TRY(cudaMemcpyAsync(ctl_out, kw.ctl, sizeof(ctl_out), cudaMemcpyDeviceToHost, st));
        HELM_CUDA_TRY(cudaMemcpyAsync(iters.data(), kw.iters, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
        HELM_CUDA_TRY(cudaMemcpyAsync(jcount.data(), kw.jcount, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
        HELM_CUDA_TRY(cudaMemcpyAsync(active.data(), kw.active, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
        HELM_CUDA_TRY(cudaMemcpyAsync(&dev_status, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
        HELM_CUDA_TRY(cudaStreamSynchronize(st));     // (thr and ctl are read before this returns)
        if (dev_status != 0) return take_device_status(p, who);
        count_launch((int)(gr->kernels * ctl_out[0]));
    }
    cycle_done = true;
    return HELM_OK;
}

// Restarted right-preconditioned flexible GMRES: x is the initial guess on entry
// (zero unless x0_given) and the iterate on exit; bnorm holds ||b|| per RHS;
// iters / relres receive the Arnoldi steps and the true relative residual
// ||b - A x|| / ||b|| at exit.  The vectors are VT (double2: all arithmetic FP64;
// float2: vector arithmetic FP32, reductions, coefficients and the least-squares
// problem FP64; the workspace arrays are allocated as double2 and hold either).
// Modified Gram-Schmidt in the persistent kernel (ortho HELM_ORTHO_MGS, FP64
// vectors), else classical Gram-Schmidt with selective reorthogonalisation, fused
// into one launch per step unless HELM_ORTHO_CGS2_SPLIT.  `who` names the caller
// in error messages.
template <typename VT>
static helm_status fgmres_core(helm_problem* p, KrylovWS& kw, long long n, int nrhs, int m, int maxit, double tol,
                               const std::vector<double>& bnorm, VT* x, bool x0_given, int ortho,
                               double* hist, const KrylovOps<VT>& ops, std::vector<int>& iters,
                               std::vector<double>& relres, const char* who, cudaStream_t st) {
    constexpr bool fp64 = std::is_same<VT, double2>::value;
    VT* const KV = reinterpret_cast<VT*>(kw.V);
    VT* const KZ = reinterpret_cast<VT*>(kw.Z);
    const long long N = n;
    helm_status s = HELM_OK;
    const int nb = kw.nblk;
    const long long vsk = (long long)nrhs * N;    // V_j of RHS k at V + j*vsk + k*N
    const int ld = m + 1;
    // modified Gram-Schmidt needs the vector to fit the persistent kernel's registers
    const int mgs_grid_n = (fp64 && ortho == HELM_ORTHO_MGS) ? mgs_grid() : 0;
    const bool use_mgs = mgs_grid_n > 0 && N <= mgs_max_n(mgs_grid_n) && kw.mgs_part != nullptr;
    // classical Gram-Schmidt: one fused launch per step when a slice of the vector per CTA
    // fits in shared memory, else the reduction kernels one by one
    const int cgs2_grid_n =
        (!use_mgs && ortho != HELM_ORTHO_CGS2_SPLIT && kw.mgs_part != nullptr && kw.restart >= m) ? cgs2_grid<VT>(N, m)
                                                                                                : 0;
    // device-driven Arnoldi loop: one graph launch per restart cycle, the steps repeated
    // by a conditional (while) node until every RHS stopped or the cycle is full; the
    // host synchronises once per cycle instead of once per step.  Needs the fused
    // Gram-Schmidt step, no residual history and no per-launch profiling events.
    const bool dev_loop = ops.dev_step && cgs2_grid_n > 0 && !hist && !p->prof_on && p->persistent != 1 &&
                          !p->dev_loop_broken && kw.ctl && kw.restart >= m;
    if (!x0_given) HELM_CUDA_TRY(cudaMemsetAsync(x, 0, (size_t)nrhs * N * sizeof(VT), st));

    std::vector<double> rn(nrhs), est(nrhs);
    std::vector<int> need(nrhs, 0);
    std::vector<int> done(nrhs, 0), active(nrhs, 0), jcount(nrhs, 0);
    iters.assign(nrhs, 0);
    relres.assign(nrhs, 0.0);
    int dev_status = 0;
    for (int k = 0; k < nrhs; ++k) done[k] = bnorm[k] == 0.0;

    bool x_zero = !x0_given;
    while (true) {
        // r = b - A x into V_0, beta = ||r||
        s = ops.residual(x, x_zero, KV);
        if (s != HELM_OK) return s;
        x_zero = false;
        launch_norm2_partial(KV, N, nrhs, N, kw.rpart, nb, st);
        launch_reduce_rows(kw.rpart, nb, nrhs, kw.rn, 1, st);
        HELM_CUDA_TRY(cudaMemcpyAsync(rn.data(), kw.rn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
        HELM_CUDA_TRY(cudaStreamSynchronize(st));
        bool any = false;
        for (int k = 0; k < nrhs; ++k) {
            relres[k] = bnorm[k] > 0 ? rn[k] / bnorm[k] : 0.0;
            if (relres[k] <= tol || iters[k] >= maxit) done[k] = 1;
            active[k] = !done[k];
            any |= active[k] != 0;
            jcount[k] = 0;
        }
        if (!any) break;
        HELM_CUDA_TRY(cudaMemcpyAsync(kw.active, active.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        // g = beta e_1, V_0 = r / beta
        {
            std::vector<double2> g0((size_t)nrhs * ld, make_double2(0, 0));
            std::vector<double> inv(nrhs);
            for (int k = 0; k < nrhs; ++k) {
                g0[(size_t)k * ld] = make_double2(rn[k], 0.0);
                inv[k] = rn[k] > 0 ? 1.0 / rn[k] : 0.0;
            }
            HELM_CUDA_TRY(cudaMemcpyAsync(kw.g, g0.data(), g0.size() * sizeof(double2), cudaMemcpyHostToDevice, st));
            HELM_CUDA_TRY(cudaMemcpyAsync(kw.invh, inv.data(), nrhs * sizeof(double), cudaMemcpyHostToDevice, st));
            launch_scale_vec(KV, N, KV, N, kw.invh, N, nrhs, kw.active, st);
            HELM_CUDA_TRY(cudaStreamSynchronize(st));    // host vectors above go out of scope
        }
        bool cycle_done = false;
        if (dev_loop) {
            s = device_cycle<VT>(p, kw, N, nrhs, m, maxit, tol, bnorm, ops, cgs2_grid_n, iters, active, jcount,
                                 cycle_done, who, st);
            if (s != HELM_OK) return s;
        }
        for (int j = 0; j < m && !cycle_done; ++j) {
            VT* Vj = KV + (long long)j * vsk;
            VT* Vn = KV + (long long)(j + 1) * vsk;
            VT* Zj = KZ + (long long)j * vsk;
            // z_j = M^{-1} v_j ; w = A z_j
            s = ops.precond(Vj, Zj);
            if (s != HELM_OK) return s;
            const double vb = (double)sizeof(VT) * N * nrhs;   // bytes of one field for all RHS
            s = ops.matvec(Zj, Vn);
            if (s != HELM_OK) return s;
            if (use_mgs) {
                // modified Gram-Schmidt, persistent kernel: h = column j of H, ||w||, v_{j+1}
                int nact = 0;
                for (int k = 0; k < nrhs; ++k) nact += active[k];
                prof_begin(p, HELM_K_ORTHO, st);
                // (FP64 vectors only: use_mgs is false for float2)
                cudaError_t e = launch_mgs(kw.V, vsk, N, reinterpret_cast<double2*>(Vn), j + 1, N, nrhs, kw.active, kw.hsum, ld,
                                           kw.rn + 3 * nrhs, kw.mgs_part, kw.mgs_bar, p->d_err, mgs_grid_n, st,
                                           p->wait_cycles);
                prof_end(p, HELM_K_ORTHO, (j + 3) * 16.0 * N * nact, st, (16.0 * (j + 1) + 4.0) * N * nact);
                if (e != cudaSuccess) return cuda_status(e, "modified Gram-Schmidt launch");
                launch_hessenberg_step(kw.H, ld, (long long)ld * m, kw.cs, kw.sn, kw.g, ld, kw.hsum, ld,
                                       kw.rn + 3 * nrhs, j, nrhs, kw.active, kw.est, kw.invh, st);
                goto step_done;
            }
            if (cgs2_grid_n > 0) {
                // classical Gram-Schmidt with selective reorthogonalisation and the Givens
                // update in one cooperative launch (short vectors)
                int nact = 0;
                for (int k = 0; k < nrhs; ++k) nact += active[k];
                prof_begin(p, HELM_K_ORTHO, st);
                cudaError_t e = launch_cgs2_step<VT>(KV, vsk, N, j, N, nrhs, kw.active, kw.hsum, ld, kw.rn + 3 * nrhs,
                                                 kw.need, kw.H, ld, (long long)ld * m, kw.cs, kw.sn, kw.g, ld, kw.est,
                                                 kw.invh, kw.mgs_part, kw.mgs_bar, p->d_err, cgs2_grid_n, st,
                                                 nullptr, 0, nullptr, nullptr, nullptr, p->wait_cycles, ops.reorth);
                prof_end(p, HELM_K_ORTHO, (2.0 * j + 5) * (double)sizeof(VT) * N * nact, st,
                         (16.0 * (j + 1) + 4.0) * N * nact);
                if (e != cudaSuccess) return cuda_status(e, "Gram-Schmidt launch");
                if (p->prof_on)
                    HELM_CUDA_TRY(cudaMemcpyAsync(need.data(), kw.need, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
                goto step_done;
            }
            // classical Gram-Schmidt with selective reorthogonalisation (coefficients in FP64)
            launch_norm2_partial(Vn, N, nrhs, N, kw.rpart, nb, st);
            launch_reduce_rows(kw.rpart, nb, nrhs, kw.rn, 0, st);                 // ||w||^2
            prof_begin(p, HELM_K_ORTHO, st);
            launch_mdot(KV, vsk, N, j + 1, Vn, N, N, nrhs, kw.active, kw.cpart, nb, st);
            prof_end(p, HELM_K_ORTHO, (j + 2) * vb, st, 8.0 * (j + 1) * N * nrhs);
            launch_reduce_cpartials(kw.cpart, nb, j + 1, kw.h1, ld, nrhs, st);
            prof_begin(p, HELM_K_ORTHO, st);
            launch_mupdate(KV, vsk, N, j + 1, nullptr, kw.h1, ld, -1.0, Vn, N, N, nrhs, kw.active, kw.rpart,
                           nb, st);
            prof_end(p, HELM_K_ORTHO, (j + 3) * vb, st, 8.0 * (j + 1) * N * nrhs + 4.0 * N * nrhs);
            launch_reduce_rows(kw.rpart, nb, nrhs, kw.rn + nrhs, 0, st);          // ||w'||^2
            count_launch();
            dgks_decide_kernel<<<(nrhs + 127) / 128, 128, 0, st>>>(kw.rn, kw.active, kw.need, nrhs, ops.reorth);
            prof_begin(p, HELM_K_ORTHO, st);
            launch_mdot(KV, vsk, N, j + 1, Vn, N, N, nrhs, kw.need, kw.cpart, nb, st);
            prof_end(p, HELM_K_ORTHO, 0.0, st);
            launch_reduce_cpartials(kw.cpart, nb, j + 1, kw.h2, ld, nrhs, st);
            prof_begin(p, HELM_K_ORTHO, st);
            launch_mupdate(KV, vsk, N, j + 1, nullptr, kw.h2, ld, -1.0, Vn, N, N, nrhs, kw.need, kw.rpart,
                           nb, st);
            prof_end(p, HELM_K_ORTHO, 0.0, st);
            launch_reduce_rows(kw.rpart, nb, nrhs, kw.rn + 2 * nrhs, 0, st);      // ||w''||^2
            count_launch();
            dgks_norm_kernel<<<(nrhs + 127) / 128, 128, 0, st>>>(kw.rn, kw.need, kw.rn + 3 * nrhs, nrhs);
            count_launch();
            add_cols_kernel<<<nrhs, 128, 0, st>>>(kw.h1, kw.h2, kw.hsum, j + 1, nrhs, ld);
            launch_hessenberg_step(kw.H, ld, (long long)ld * m, kw.cs, kw.sn, kw.g, ld, kw.hsum, ld, kw.rn + 3 * nrhs, j,
                                   nrhs, kw.active, kw.est, kw.invh, st);
            launch_scale_vec(Vn, N, Vn, N, kw.invh, N, nrhs, kw.active, st);
            if (p->prof_on)
                HELM_CUDA_TRY(cudaMemcpyAsync(need.data(), kw.need, nrhs * sizeof(int), cudaMemcpyDeviceToHost, st));
        step_done:
            HELM_CUDA_TRY(cudaGetLastError());
            HELM_CUDA_TRY(cudaMemcpyAsync(est.data(), kw.est, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
            HELM_CUDA_TRY(cudaMemcpyAsync(&dev_status, p->d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
            HELM_CUDA_TRY(cudaStreamSynchronize(st));
            if (dev_status != 0) return take_device_status(p, who);   // a bounded device wait expired
            if (p->prof_on && !use_mgs) {
                // the second Gram-Schmidt pass ran for the RHS that needed it
                int nre = 0;
                for (int k = 0; k < nrhs; ++k) nre += need[k];
                prof_add(p, HELM_K_ORTHO, (2.0 * j + 5) * 16.0 * N * nre, (16.0 * (j + 1) + 4.0) * N * nre);
            }
            bool still = false, changed = false;
            for (int k = 0; k < nrhs; ++k) {
                if (!active[k]) continue;
                if (hist && iters[k] < maxit) hist[(size_t)k * maxit + iters[k]] = est[k] / bnorm[k];
                ++iters[k];
                jcount[k] = j + 1;
                if (est[k] <= tol * bnorm[k] || iters[k] >= maxit || !std::isfinite(est[k])) {
                    active[k] = 0;
                    changed = true;
                }
                still |= active[k] != 0;
            }
            if (!still) break;
            // the host array is next written after the next step's synchronisation, which
            // orders this copy before it
            if (changed)
                HELM_CUDA_TRY(cudaMemcpyAsync(kw.active, active.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        }
        // u += Z y with y = R^{-1} g
        HELM_CUDA_TRY(cudaMemcpyAsync(kw.jcount, jcount.data(), nrhs * sizeof(int), cudaMemcpyHostToDevice, st));
        launch_hessenberg_solve(kw.H, ld, (long long)ld * m, kw.g, ld, kw.jcount, kw.y, ld, nrhs, st);
        launch_mupdate(KZ, vsk, N, m, kw.jcount, kw.y, ld, 1.0, x, N, N, nrhs, nullptr, nullptr, nb, st);
        HELM_CUDA_TRY(cudaGetLastError());
        HELM_CUDA_TRY(cudaStreamSynchronize(st));
    }
    return take_device_status(p, who);
}

// ----------------------------------------------- interface Krylov preconditioner
// z = M^{-1} r with the interface problem solved by Krylov iterations, the
// paper's own formulation (Sections 3-5: GMRES on (I - S) g = b, preconditioned
// by the SP or BSP sweep): liftings (source r, no incoming data) give b; g is
// the FGMRES(inner_restart) iterate after at most inner_maxit steps or at
// relative residual inner_tol, with the sweep of the schedule as its
// preconditioner; the reconstruction (source r, incoming g) gives z.  The
// interface vectors are FP64; S and the sweep run in the precision of the
// factors.  With an exact interface solve M^{-1} = A^{-1}.
template <typename R, typename VT>
static helm_status run_precond_iface_t(helm_problem* p, int sched, const double2* r, double2* z, int nrhs,
                                       const helm_opts& o, cudaStream_t st) {
    NvtxRange nvtx("interface FGMRES");
    using T = Cx<R>;
    const std::vector<StageDesc>& stg = p->sched[sched];
    if (stg.size() < 2 || p->ntrace == 0) return run_precond(p, sched, r, z, nrhs, st);   // one subdomain
    helm_status s = ensure_pc_ws(p, nrhs);
    if (s != HELM_OK) return s;
    s = tune_shape(p, nrhs, st);
    if (s != HELM_OK) return s;
    s = tune_stage(p, r, nrhs, st);
    if (s != HELM_OK) return s;
    const long long nt = p->ntrace;
    s = ensure_kw(p->kwi, nrhs, o.inner_restart, nt, true);
    if (s != HELM_OK) return s;
    // typed views of the interface workspace (allocated by ensure_kw just above)
    VT* const kb = reinterpret_cast<VT*>(p->kwi.b);      // interface right-hand side
    VT* const kx = reinterpret_cast<VT*>(p->kwi.x);      // interface iterate
    const PcWork w{{p->d_trace[0], p->d_trace[1], p->d_trace[2], p->d_trace[3]}, p->d_yws, p->d_pc_norm,
                   p->d_pc_partial, p->d_escr, p->d_r64};
    T* tB = (T*)w.trace[BUF_B];
    T* tX = (T*)w.trace[BUF_X];
    T* tY = (T*)w.trace[BUF_Y];
    const long long tot = nt * nrhs;
    const PcCtx cx = precond_prologue<R>(p, w, r, nrhs, st);
    // b: outgoing data of the liftings
    s = p->habc ? habc_lifting_t<R>(p, w, cx, stg.front(), r, nrhs, st) : run_stage_t<R>(p, w, cx, stg.front(), r, z, nrhs, st);
    if (s != HELM_OK) return s;
    launch_trace_to<T, VT>(tB, nullptr, 1, kb, tot, st);
    // (I - S) v: one interface stage over every subdomain writes S v - v into B
    StageDesc sS = stg.front();
    sS.iface = 1; sS.src = 0; sS.in0 = BUF_X; sS.in1 = BUF_NONE; sS.mask = 15;
    sS.dst = BUF_B; sS.dst2 = BUF_NONE; sS.base = BUF_NONE; sS.sub = BUF_X; sS.final_ = 0;
    KrylovOps<VT> ops;
    // The interface iteration stops at a loose relative residual (1e-2 by default) and the
    // outer FP64 FGMRES corrects whatever it leaves, so its basis needs far less than
    // working-precision orthogonality: the second Gram-Schmidt pass runs only when the
    // first cancelled more than ~68 % of ||w|| (||w'||^2 < ||w||^2 / 10; a factor of
    // at most sqrt(10) on the rounding of the new vector's projections).
    ops.reorth = 0.1;
    // the interface stages read and write only the trace buffers: captured once as graphs
    // (tags: 2 sched = the sweep, 2 sched + 1 = S)
    ops.matvec = [&](const VT* v, VT* wv) -> helm_status {
        launch_trace_from<VT, T>(v, tX, (T*)nullptr, tot, st);
        helm_status q = run_captured(p, 2 * sched + 1, nrhs, st, [&](cudaStream_t cs) {
            return run_stage_t<R>(p, w, cx, sS, r, z, nrhs, cs);
        });
        if (q != HELM_OK) return q;
        launch_trace_to<T, VT>(tB, nullptr, -1, wv, tot, st);
        return HELM_OK;
    };
    // the sweep of the schedule (its stages between lifting and reconstruction) on v:
    // input in B (and X, where SP propagates from), result X (SP) or X + Y (BSP)
    ops.precond = [&](const VT* v, VT* zv) -> helm_status {
        launch_trace_from<VT, T>(v, tB, tX, tot, st);
        helm_status q = HELM_OK;
        if (run_sweep_persistent<R>(p, w, sched, nrhs, st, q)) {
            if (q != HELM_OK) return q;
            launch_trace_to<T, VT>(tX, is_bsp(sched) ? tY : (T*)nullptr, 1, zv, tot, st);
            return HELM_OK;
        }
        q = run_captured(p, 2 * sched, nrhs, st, [&](cudaStream_t cs) {
            for (size_t i = 1; i + 1 < stg.size(); ++i) {
                helm_status q2 = run_stage_t<R>(p, w, cx, stg[i], r, z, nrhs, cs);
                if (q2 != HELM_OK) return q2;
            }
            return HELM_OK;
        });
        if (q != HELM_OK) return q;
        launch_trace_to<T, VT>(tX, is_bsp(sched) ? tY : (T*)nullptr, 1, zv, tot, st);
        return HELM_OK;
    };
    // one Arnoldi step with the slot read on the device (*dj): the same kernels as
    // precond + matvec above, launched directly (this runs under a capture)
    // the sweep of one step: its stage launches, or the dependency-driven persistent sweep
    auto sweep_stages = [&](cudaStream_t cs) -> helm_status {
        helm_status q = HELM_OK;
        if (p->persistent == 2 && run_sweep_persistent<R>(p, w, sched, nrhs, cs, q)) return q;
        for (size_t i = 1; i + 1 < stg.size(); ++i) {
            q = run_stage_t<R>(p, w, cx, stg[i], r, z, nrhs, cs);
            if (q != HELM_OK) return q;
        }
        return HELM_OK;
    };
    if (p->persistent != 1 && std::is_same<T, VT>::value) {
        // vectors in the trace buffers' type: the step keeps its data in the trace
        // buffers (the Gram-Schmidt step reads S v - v from B and writes the next input
        // into B and X), one kernel between the sweep and S forms z_j
        ops.dev_prologue = [&](cudaStream_t cs, VT* V) -> helm_status {
            launch_trace_from<VT, T>(V, tB, tX, tot, cs);
            return HELM_OK;
        };
        ops.dev_step = [&](cudaStream_t cs, VT* V, VT* Z, long long vsk, const int* dj) -> helm_status {
            (void)V;
            helm_status q0 = sweep_stages(cs);
            if (q0 != HELM_OK) return q0;
            // z_j = X (+ Y) into Z slot j and into X, the input of S
            launch_trace_to<T, VT>(tX, is_bsp(sched) ? tY : (T*)nullptr, 1, Z, tot, cs, dj, 0, vsk,
                                   reinterpret_cast<VT*>(tX));
            return run_stage_t<R>(p, w, cx, sS, r, z, nrhs, cs);
        };
        ops.dev_w_src = reinterpret_cast<VT*>(tB);
        ops.dev_v_out1 = reinterpret_cast<VT*>(tB);
        ops.dev_v_out2 = reinterpret_cast<VT*>(tX);
        ops.dev_tag = 2 * sched + 1 + 16 * p->persistent;
    } else if (p->persistent != 1) {
        ops.dev_tag = 2 * sched + 16 * p->persistent;
        ops.dev_step = [&](cudaStream_t cs, VT* V, VT* Z, long long vsk, const int* dj) -> helm_status {
            launch_trace_from<VT, T>(V, tB, tX, tot, cs, dj, 0, vsk);
            helm_status q0 = sweep_stages(cs);
            if (q0 != HELM_OK) return q0;
            launch_trace_to<T, VT>(tX, is_bsp(sched) ? tY : (T*)nullptr, 1, Z, tot, cs, dj, 0, vsk);
            launch_trace_from<VT, T>(Z, tX, (T*)nullptr, tot, cs, dj, 0, vsk);
            helm_status q = run_stage_t<R>(p, w, cx, sS, r, z, nrhs, cs);
            if (q != HELM_OK) return q;
            launch_trace_to<T, VT>(tB, nullptr, -1, V, tot, cs, dj, 1, vsk);
            return HELM_OK;
        };
    }
    ops.residual = [&](const VT* x, bool x_zero, VT* rv) -> helm_status {
        if (x_zero) {
            HELM_CUDA_TRY(cudaMemcpyAsync(rv, kb, (size_t)tot * sizeof(VT), cudaMemcpyDeviceToDevice, st));
            return HELM_OK;
        }
        helm_status q = ops.matvec(x, rv);
        if (q != HELM_OK) return q;
        launch_sub<VT>(kb, rv, rv, tot, st);
        return HELM_OK;
    };
    std::vector<double> bnorm(nrhs);
    launch_norm2_partial(kb, nt, nrhs, nt, p->kwi.rpart, p->kwi.nblk, st);
    launch_reduce_rows(p->kwi.rpart, p->kwi.nblk, nrhs, p->kwi.rn, 1, st);
    HELM_CUDA_TRY(cudaMemcpyAsync(bnorm.data(), p->kwi.rn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    HELM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<int> it;
    std::vector<double> rr;
    // the first application of a call may record the interface residual history
    double* ihist = (o.inner_hist && !p->inner_hist_taken) ? o.inner_hist : nullptr;
    if (ihist) p->inner_hist_taken = true;
    s = fgmres_core<VT>(p, p->kwi, nt, nrhs, o.inner_restart, o.inner_maxit, o.inner_tol, bnorm, kx, false,
                    o.ortho == HELM_ORTHO_CGS2_SPLIT ? HELM_ORTHO_CGS2_SPLIT : HELM_ORTHO_CGS2, ihist, ops, it, rr,
                    "gmres_solve (interface iterations)", st);
    if (s != HELM_OK) return s;
    p->inner_steps += it.empty() ? 0 : *std::max_element(it.begin(), it.end());
    // reconstruction with the incoming data g
    launch_trace_from<VT, T>(kx, tX, (T*)nullptr, tot, st);
    StageDesc sR = stg.back();
    sR.in0 = BUF_X; sR.in1 = BUF_NONE;
    if (p->habc) return habc_recon_t<R>(p, w, cx, sR, BUF_X, BUF_NONE, BUF_B, BUF_Y, r, z, nrhs, st);
    return run_stage_t<R>(p, w, cx, sR, r, z, nrhs, st);
}

static helm_status run_precond_iface(helm_problem* p, int sched, const double2* r, double2* z, int nrhs,
                                     const helm_opts& o, cudaStream_t st) {
    // interface vectors in the factors' precision unless inner_fp64
    if (p->prec != HELM_PREC_C64) return run_precond_iface_t<double, double2>(p, sched, r, z, nrhs, o, st);
    return o.inner_fp64 ? run_precond_iface_t<float, double2>(p, sched, r, z, nrhs, o, st)
                        : run_precond_iface_t<float, float2>(p, sched, r, z, nrhs, o, st);
}

// FGMRES on A u = h^2 f for one chunk of right-hand sides
static helm_status gmres_impl(helm_problem* p, const double2* f, double2* u, int nrhs, const helm_opts& o,
                              helm_info* info, cudaStream_t st) {
    const long long N = p->N();
    helm_status s = ensure_kw(p->kw, nrhs, o.restart, N, false);
    if (s != HELM_OK) return s;
    s = ensure_pc_ws(p, nrhs);
    if (s != HELM_OK) return s;
    s = tune_shape(p, nrhs, st);
    if (s != HELM_OK) return s;
    const double h2 = p->h * p->h;
    // ||h^2 f||
    std::vector<double> bnorm(nrhs);
    launch_norm2_partial(f, N, nrhs, N, p->kw.rpart, p->kw.nblk, st);
    launch_reduce_rows(p->kw.rpart, p->kw.nblk, nrhs, p->kw.rn, 1, st);
    HELM_CUDA_TRY(cudaMemcpyAsync(bnorm.data(), p->kw.rn, nrhs * sizeof(double), cudaMemcpyDeviceToHost, st));
    HELM_CUDA_TRY(cudaStreamSynchronize(st));
    for (auto& b : bnorm) b *= h2;
    KrylovOps<double2> ops;
    ops.residual = [&](const double2* x, bool, double2* rv) -> helm_status {
        launch_residual(p->d_adiag, p->nx, p->ny, f, h2, x, rv, nrhs, nullptr, p->kw.rpart, p->kw.nblk, st);
        return HELM_OK;
    };
    ops.matvec = [&](const double2* zv, double2* wv) -> helm_status {
        prof_begin(p, HELM_K_MATVEC, st);
        launch_matvec(p->d_adiag, p->nx, p->ny, zv, wv, nrhs, st);
        prof_end(p, HELM_K_MATVEC, 48.0 * N * nrhs + 16.0 * N, st, 16.0 * N * nrhs);
        return HELM_OK;
    };
    ops.precond = [&](const double2* v, double2* zv) -> helm_status {
        if (o.inner_maxit > 0) return run_precond_iface(p, o.sched, v, zv, nrhs, o, st);
        return o.use_graph ? run_precond_graph(p, o.sched, v, zv, nrhs, st) : run_precond(p, o.sched, v, zv, nrhs, st);
    };
    std::vector<int> iters;
    std::vector<double> relres;
    p->persistent = o.persistent;
    p->wait_cycles = o.wait_cycles;
    p->inner_hist_taken = false;
    s = fgmres_core(p, p->kw, N, nrhs, o.restart, o.maxit, o.tol, bnorm, u, o.x0_given != 0, o.ortho,
                    o.hist, ops, iters, relres, "gmres_solve", st);
    p->persistent = 0;
    p->wait_cycles = 0;
    if (s != HELM_OK) return s;
    bool ok = true;
    for (int k = 0; k < nrhs; ++k) {
        if (info) { info[k].iters = iters[k]; info[k].relres = relres[k]; }
        if (relres[k] > o.tol) ok = false;
    }
    if (!ok) {
        set_error("gmres_solve: tolerance not reached within maxit");
        return HELM_ERR_NO_CONVERGENCE;
    }
    return HELM_OK;
}

extern "C" helm_status gmres_solve(helm_problem* p, const helm_c128* f, helm_c128* u, int nrhs, const helm_opts* opts,
                                   helm_info* info, void* stream) {
    NvtxRange nvtx("gmres_solve");
    if (!p) return arg_error("gmres_solve: NULL handle");
    if (!p->factored) { set_error("gmres_solve: call precond_factor first"); return HELM_ERR_STATE; }
    if (nrhs < 0) return arg_error("gmres_solve: nrhs < 0");
    if (nrhs == 0) return HELM_OK;
    if (!f || !u) return arg_error("gmres_solve: NULL array");
    const size_t vb = (size_t)p->N() * nrhs * sizeof(double2);
    HcCall hcc{{f, vb}, {u, vb}};
    helm_opts o;
    helm_default_opts(&o);
    if (opts) o = *opts;
    if (o.restart < 1 || o.restart > 500) return arg_error("gmres_solve: restart must be in 1..500");
    if (o.maxit < 1) return arg_error("gmres_solve: maxit must be >= 1");
    if (!(o.tol > 0)) return arg_error("gmres_solve: tol must be > 0");
    if ((o.sched < 0 || o.sched >= HELM_NSCHED)) return arg_error("gmres_solve: unknown schedule");
    if (o.ortho != HELM_ORTHO_MGS && o.ortho != HELM_ORTHO_CGS2 && o.ortho != HELM_ORTHO_CGS2_SPLIT)
        return arg_error("gmres_solve: unknown ortho");
    if (o.inner_maxit < 0) return arg_error("gmres_solve: inner_maxit must be >= 0");
    if (o.persistent < 0 || o.persistent > 2) return arg_error("gmres_solve: persistent must be 0, 1 or 2");
    if (o.inner_fp64 != 0 && o.inner_fp64 != 1) return arg_error("gmres_solve: inner_fp64 must be 0 or 1");
    if (o.wait_cycles < 0) return arg_error("gmres_solve: wait_cycles must be >= 0");
    if (o.inner_maxit > 0 && (o.inner_restart < 1 || o.inner_restart > 500))
        return arg_error("gmres_solve: inner_restart must be in 1..500");
    if (o.inner_maxit > 0 && !(o.inner_tol > 0)) return arg_error("gmres_solve: inner_tol must be > 0");
    // Right-hand sides are solved in chunks of equal size whose workspace fits in 80 % of
    // the device memory that is free now (the workspace already allocated counts as free):
    // per RHS the volume Krylov fields ((2 restart + 1) complex128 vectors, and two more),
    // the interface Krylov fields of the nested solve ((2 inner_restart + 1) trace
    // vectors), and the preconditioner's interface buffers, solve workspace and scaled
    // source.
    const long long N = p->N();
    size_t freeb = 0, totalb = 0;
    HELM_CUDA_TRY(cudaMemGetInfo(&freeb, &totalb));
    const size_t pelem = p->prec == HELM_PREC_C64 ? sizeof(float2) : sizeof(double2);
    const size_t nt = (size_t)std::max<long long>(p->ntrace, 0);
    auto pc_per_rhs = [&]() {
        return (size_t)(p->habc ? 4 : 3) * nt * pelem + (size_t)N * pelem + (size_t)N * sizeof(float2) +
               (size_t)2 * p->etot * sizeof(float2);
    };
    const size_t held = (size_t)p->kw.nrhs * ((size_t)2 * p->kw.restart + 1) * N * sizeof(double2) +
                        (size_t)p->kwi.nrhs * ((size_t)2 * p->kwi.restart + 1) * nt * sizeof(double2) +
                        (size_t)p->ws_nrhs * pc_per_rhs();
    const size_t per_rhs = ((size_t)2 * o.restart + 1) * N * sizeof(double2) + (size_t)N * 2 * sizeof(double2) +
                           (o.inner_maxit > 0 ? ((size_t)2 * o.inner_restart + 1) * nt * sizeof(double2) : 0) +
                           pc_per_rhs();
    long long fit = (long long)((0.8 * (double)(freeb + held)) / (double)per_rhs);
    if (p->sopts.device_budget > 0) {
        // within what the factors leave of the handle's budget
        const double left = (double)p->sopts.device_budget -
                            (double)(p->X_bytes + p->XT_bytes + p->K_bytes + (p->d_Kp ? sym_bytes(p) : 0));
        fit = std::min(fit, (long long)(std::max(0.0, left) / (double)per_rhs));
        if (fit < 1) {
            set_error("gmres_solve: the Krylov workspace of one right-hand side does not fit in the device budget");
            return HELM_ERR_OOM;
        }
    }
    if (fit < 1) {
        set_error("gmres_solve: the Krylov workspace of one right-hand side does not fit in device memory; "
                  "lower the restart length");
        return HELM_ERR_OOM;
    }
    // as many chunks as needed, all of (nearly) the same size: a small last chunk would
    // fall below the tensor-core threshold and repeat the nested iterations for few RHS
    const long long nchunks = (nrhs + std::min<long long>(fit, nrhs) - 1) / std::min<long long>(fit, nrhs);
    const int chunk = (int)((nrhs + nchunks - 1) / nchunks);
    helm_status worst = HELM_OK;
    for (int k0 = 0; k0 < nrhs; k0 += chunk) {
        const int nk = std::min(chunk, nrhs - k0);
        if (chunk < nrhs && p->kw.nrhs > nk) free_krylov(p);        // never hold more than one chunk
        const helm_status s = gmres_impl(p, (const double2*)f + (size_t)k0 * N, (double2*)u + (size_t)k0 * N, nk, o,
                                         info ? info + k0 : nullptr, (cudaStream_t)stream);
        if (s == HELM_ERR_NO_CONVERGENCE) worst = s;
        else if (s != HELM_OK) return s;
    }
    if (worst != HELM_OK) set_error("gmres_solve: tolerance not reached within maxit");
    return worst;
}

// ----------------------------------------------------------------- adjoint
extern "C" helm_status misfit_grad(helm_problem* p, const helm_c128* f, int nsrc, const int* rec_idx, int nrec,
                                   const helm_c128* d, const helm_opts* opts, double* misfit, double* grad_m2,
                                   helm_c128* u_out, void* stream) {
    NvtxRange nvtx("misfit_grad");
    if (!p) return arg_error("misfit_grad: NULL handle");
    if (!p->factored) { set_error("misfit_grad: call precond_factor first"); return HELM_ERR_STATE; }
    if (nsrc < 1 || nrec < 1) return arg_error("misfit_grad: nsrc and nrec must be >= 1");
    if (!f || !rec_idx || !d || !misfit || !grad_m2) return arg_error("misfit_grad: NULL array");
    cudaStream_t st = (cudaStream_t)stream;
    const long long N = p->N();
    HcCall hcc{{f, (size_t)nsrc * N * sizeof(double2)}, {rec_idx, (size_t)nrec * sizeof(int)},
               {d, (size_t)nsrc * nrec * sizeof(double2)}, {grad_m2, (size_t)N * sizeof(double)},
               {u_out, (size_t)nsrc * N * sizeof(double2)}};
    // receivers must be valid nodes
    {
        std::vector<int> r(nrec);
        HELM_CUDA_TRY(cudaMemcpy(r.data(), rec_idx, nrec * sizeof(int), cudaMemcpyDefault));
        for (int v : r)
            if (v < 0 || v >= N) return arg_error("misfit_grad: receiver index out of range");
    }
    if (p->aw_nsrc < nsrc || p->aw_nrec < nrec) {
        free_adj(p);
        cudaError_t e = cudaSuccess;
        auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
        chk(dalloc(p->d_res, (size_t)nsrc * nrec));
        chk(dalloc(p->d_fadj, (size_t)nsrc * N));
        chk(dalloc(p->d_U, (size_t)nsrc * N));
        chk(dalloc(p->d_L, (size_t)nsrc * N));
        chk(dalloc(p->d_jpart, (size_t)nsrc));
        if (e != cudaSuccess) { free_adj(p); return cuda_status(e, "allocating the adjoint workspace"); }
        p->aw_nsrc = nsrc;
        p->aw_nrec = nrec;
    }
    helm_opts o;
    helm_default_opts(&o);
    if (opts) o = *opts;
    o.x0_given = 0;
    std::vector<helm_info> inf(nsrc);
    double2* U = u_out ? (double2*)u_out : p->d_U;
    helm_status s = gmres_solve(p, f, (helm_c128*)U, nsrc, &o, inf.data(), stream);
    if (s != HELM_OK) return s;
    launch_receiver_residual(U, N, rec_idx, nrec, (const double2*)d, nsrc, p->d_res, p->d_jpart, st);
    HELM_CUDA_TRY(cudaMemsetAsync(p->d_fadj, 0, (size_t)nsrc * N * sizeof(double2), st));
    launch_adjoint_rhs(p->d_res, rec_idx, nrec, nsrc, N, 1.0 / (p->h * p->h), p->d_fadj, st);
    s = gmres_solve(p, (helm_c128*)p->d_fadj, (helm_c128*)p->d_L, nsrc, &o, inf.data(), stream);
    if (s != HELM_OK) return s;
    launch_gradient(U, p->d_L, p->d_m2, p->nx, p->ny, p->h, p->omega, nsrc, grad_m2, st);
    HELM_CUDA_TRY(cudaGetLastError());
    launch_reduce_rows(p->d_jpart, nsrc, 1, p->kw.rn, 0, st);
    HELM_CUDA_TRY(cudaMemcpyAsync(misfit, p->kw.rn, sizeof(double), cudaMemcpyDeviceToHost, st));
    HELM_CUDA_TRY(cudaStreamSynchronize(st));
    return HELM_OK;
}
