// best_vegas_iteration_noalloc: one VEGAS iteration of one task for callers
// that cannot allocate device memory (see include/best.h).
//
// Every piece of device memory this path needs beyond the caller's inputs
// and outputs -- time state, spline tables, the task's descriptors and
// constants, the work partition and the per-CTA partial records of the
// sample kernel -- lives in one file-scope __device__ array, g_scratch.  Its
// device address is obtained once per device with cudaGetSymbolAddress (the
// symbol itself is only a host-side stand-in).  The kernels are the ones the
// context path uses; nothing here calls cudaMalloc or cudaFree.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "internal.cuh"
#include "philox.cuh"

namespace best {
__global__ void spline_build_kernel(Geometry, const double*, int, const double*, TimeState*, SpeciesConst*,
                                    double*, double*, float*);
__global__ void prepare_kernel(Geometry, const SideDesc*, const TaskDesc*, const double*, const double*,
                               const TimeState*, const double*, TaskConst*, TaskAcc*, int, const double*,
                               const SpeciesConst*, SegConst32*);
__global__ void map32_kernel(Geometry, const TaskDesc*, int, const double*, float2*);
void* eval_kernel_ptr_f32(int nmax);
void* eval_kernel_ptr_f64(int nmax);
best_status check_config(const best_config* cfg);
best_status report(best_status st, const char* msg);
bool describe_task(const best_config* cfg, int32_t task, SideDesc* sd, TaskDesc* td);
}  // namespace best

using namespace best;

namespace {

// Limits of this path, fixed by the size of g_scratch.
constexpr int kMaxGrid = 512;
constexpr int kMaxBins = 64;
constexpr int kMaxCtas = 512;
constexpr int kRecord = 2 + kMaxDim * kMaxBins;          // doubles per partial record
constexpr size_t kAlign = 256;

constexpr size_t up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets inside g_scratch.
constexpr size_t kOffTs = 0;
constexpr size_t kOffSc = up(kOffTs + sizeof(TimeState));
constexpr size_t kOffSide = up(kOffSc + sizeof(SpeciesConst) * BEST_MAX_SPECIES);
constexpr size_t kOffTask = up(kOffSide + sizeof(SideDesc));
constexpr size_t kOffTconst = up(kOffTask + sizeof(TaskDesc));
constexpr size_t kOffTc32 = up(kOffTconst + sizeof(TaskConst));
constexpr size_t kOffMap32 = up(kOffTc32 + sizeof(SegConst32));
constexpr size_t kOffAcc = up(kOffMap32 + sizeof(float2) * kMaxDim * kMaxBins);
constexpr size_t kOffPrev = up(kOffAcc + sizeof(TaskAcc));
constexpr size_t kOffKnots = up(kOffPrev + sizeof(double));
constexpr size_t kOffKnots32 = up(kOffKnots + sizeof(double) * kMaxGrid);
constexpr size_t kOffFgrid = up(kOffKnots32 + sizeof(float) * kMaxGrid);
constexpr size_t kOffCoef64 = up(kOffFgrid + sizeof(double) * BEST_MAX_SPECIES * kMaxGrid);
constexpr size_t kOffCoef32 = up(kOffCoef64 + sizeof(double) * BEST_MAX_SPECIES * (kMaxGrid - 1) * 4);
constexpr size_t kOffSegs = up(kOffCoef32 + sizeof(float) * BEST_MAX_SPECIES * (kMaxGrid - 1) * 4);
constexpr size_t kOffCtaSeg = up(kOffSegs + sizeof(Segment) * kMaxCtas);
constexpr size_t kOffPart = up(kOffCtaSeg + sizeof(int32_t) * (kMaxCtas + 1));
constexpr size_t kScratchBytes = up(kOffPart + sizeof(double) * static_cast<size_t>(kMaxCtas) * kRecord);

// Per-device set-up: the device address of g_scratch (looked up under a
// lock, so that two host threads making their first call on one device do
// not both write the slot).
constexpr int kMaxDevices = 64;
unsigned char* g_base[kMaxDevices] = {};
std::mutex g_base_lock;

}  // namespace

// The scratch array (about 3.5 MiB), held by every device that loads the library.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

namespace {

struct SetupArgs {
    Geometry g;
    TimeState ts;
    SpeciesConst sc[BEST_MAX_SPECIES];
    SideDesc sd;
    TaskDesc td;
    int32_t ctas;
    int64_t groups;
};

// Writes the descriptors, the grid, the time state and the partition of the
// task's sample groups over the CTAs into the scratch array, and clears the
// previous-estimate slot (the adaptive scale starts from f_obs).  The task's
// descriptors sit at index 0 of the scratch arrays, so every segment names
// task 0; the Philox stream is keyed by the descriptor's gid, which holds
// the task's id in the whole grid's numbering.
__global__ void noalloc_setup_kernel(SetupArgs A, unsigned char* base) {
    const int tid = threadIdx.x;
    const Geometry& g = A.g;
    double* knots = reinterpret_cast<double*>(base + kOffKnots);
    float* knots32 = reinterpret_cast<float*>(base + kOffKnots32);
    for (int j = tid; j < g.n_grid; j += blockDim.x) {
        double q;
        if (j == 0) q = g.q_min;
        else if (j == g.n_grid - 1) q = g.q_max;
        else if (g.log_spaced) q = g.q_min * pow(g.q_max / g.q_min, static_cast<double>(j) / (g.n_grid - 1));
        else q = g.q_min + (g.q_max - g.q_min) * j / (g.n_grid - 1);
        knots[j] = q;
        knots32[j] = static_cast<float>(q);
    }
    Segment* segs = reinterpret_cast<Segment*>(base + kOffSegs);
    int32_t* cta_seg = reinterpret_cast<int32_t*>(base + kOffCtaSeg);
    for (int b = tid; b < A.ctas; b += blockDim.x) {
        Segment s{};
        s.task = 0;
        s.g0 = A.groups * b / A.ctas;
        s.g1 = A.groups * (b + 1) / A.ctas;
        s.part = static_cast<int64_t>(b) * kRecord;
        segs[b] = s;
        cta_seg[b] = b;
    }
    if (tid == 0) {
        cta_seg[A.ctas] = A.ctas;
        *reinterpret_cast<TimeState*>(base + kOffTs) = A.ts;
        SpeciesConst* sc = reinterpret_cast<SpeciesConst*>(base + kOffSc);
        for (int s = 0; s < g.n_species; ++s) sc[s] = A.sc[s];
        *reinterpret_cast<SideDesc*>(base + kOffSide) = A.sd;
        *reinterpret_cast<TaskDesc*>(base + kOffTask) = A.td;
        *reinterpret_cast<double*>(base + kOffPrev) = 0.0;
    }
}

// Sums the task's partial records in CTA order and scales them back to the
// weight's units: out[0] = sum w, out[1] = sum w^2, out[2 + d*nb + b] =
// sum of w^2 over the samples in increment b of dimension d.  When the
// spline build flagged the grid values (a value <= 0 or not finite: the
// time state's sticky error), every output is NaN instead.
__global__ void noalloc_reduce_kernel(const unsigned char* base, int ctas, int L, double* out) {
    const TaskConst& c = *reinterpret_cast<const TaskConst*>(base + kOffTconst);
    const TimeState& ts = *reinterpret_cast<const TimeState*>(base + kOffTs);
    const double* part = reinterpret_cast<const double*>(base + kOffPart);
    const double sc = c.K * c.scale;
    const bool bad = ts.error != 0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int b = 0; b < ctas; ++b) v += part[static_cast<int64_t>(b) * kRecord + k];
        out[k] = bad ? __longlong_as_double(0x7FF8000000000000LL) : (k == 0 ? v * sc : v * sc * sc);
    }
}

int group_size(int D, bool f32) {
    const int per = f32 ? 4 : 2;
    int a = D, b = per;
    while (b) { const int t = a % b; a = b; b = t; }
    return per / a;
}

}  // namespace

extern "C" best_status best_vegas_iteration_noalloc(const best_config* cfg, int32_t task, const double* f_dev,
                                                    double t, const double* edges_dev, uint32_t iteration,
                                                    uint32_t call, double* out_dev, void* stream) {
    best_status vs = check_config(cfg);
    if (vs != BEST_OK) return vs;
    if (!f_dev || !edges_dev || !out_dev) return report(BEST_ERR_INVALID, "f, edges and out must not be NULL");
    if (!std::isfinite(t)) return report(BEST_ERR_INVALID, "t must be finite");
    if (cfg->grid.n > kMaxGrid) return report(BEST_ERR_INVALID, "noalloc: grid.n exceeds 512");
    SideDesc sd;
    TaskDesc td;
    if (task < 0 || !describe_task(cfg, task, &sd, &td)) return report(BEST_ERR_INVALID, "noalloc: task out of range");
    if (td.nbins > kMaxBins) return report(BEST_ERR_INVALID, "noalloc: nbins exceeds 64");
    if (cfg->processes[sd.process].strat)
        return report(BEST_ERR_INVALID, "noalloc: stratified sampling is not supported here");
    if (sd.me_on)
        return report(BEST_ERR_INVALID, "noalloc: s-dependent matrix elements are not supported here");
    const bool f32 = cfg->precision == BEST_FP32;

    // Set-up once per device: the device address of the scratch array.
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return report(BEST_ERR_CUDA, "noalloc: no usable CUDA device");
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_base_lock);
        if (!g_base[dev]) {
            void* p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) return report(BEST_ERR_CUDA, "noalloc: cudaGetSymbolAddress failed");
            g_base[dev] = static_cast<unsigned char*>(p);
        }
        base = g_base[dev];
    }

    // Geometry of this single task.
    const int D = td.dim, nb = td.nbins, n = cfg->grid.n, S = cfg->n_species;
    Geometry g{};
    g.n_grid = n;
    g.log_spaced = cfg->grid.log_spaced ? 1 : 0;
    g.q_min = cfg->grid.q_min;
    g.q_max = cfg->grid.q_max;
    g.log_step = g.log_spaced ? std::log(g.q_max / g.q_min) / (n - 1) : (g.q_max - g.q_min) / (n - 1);
    g.inv_step = 1.0 / (g.log_spaced ? g.log_step / 0.6931471805599453 : g.log_step);
    g.lq0_step = g.log_spaced ? std::log2(g.q_min) * g.inv_step : 0.0;
    g.n_species = S;
    g.n_tasks = 1;
    g.n_side = 1;
    g.map_stride = D * (nb + 1);
    g.nbins_max = nb;
    g.expansion = cfg->expansion ? 1 : 0;
    g.a0 = cfg->a0;
    g.t0 = cfg->t0;
    g.e_cut = cfg->e_cut;
    g.eps_dt = cfg->eps_dt;
    g.seed = cfg->seed;
    g.tail_points = cfg->tail_points;
    g.precision = cfg->precision;

    // Launch shape of the sample kernel (shared memory limit raised, never lowered).
    void* fn = f32 ? eval_kernel_ptr_f32(sd.n) : eval_kernel_ptr_f64(sd.n);
    const size_t rs = f32 ? 4 : 8;
    const size_t spl = static_cast<size_t>(S) * 4 * (n - 1) + n;
    const size_t map_elems = static_cast<size_t>(kMaxDim) * nb;
    const size_t hist_elems = static_cast<size_t>(kThreads / 32) * map_elems;
    const size_t smem = rs * ((spl + 3) & ~size_t(3)) + 2 * rs * map_elems + rs * ((hist_elems + 3) & ~size_t(3)) +
                        2 * 32 * sizeof(double) +
                        (f32 ? sizeof(float) * (kThreads / 32) * kQueueSlots * queue_words(sd.n) : 0);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return report(BEST_ERR_CUDA, "noalloc: kernel query failed");
    if (static_cast<size_t>(fa.maxDynamicSharedSizeBytes) < smem &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
        return report(BEST_ERR_INVALID, "noalloc: spline and map tables exceed shared memory");
    int occ = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kThreads, smem) != cudaSuccess || occ < 1 ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return report(BEST_ERR_CUDA, "noalloc: sample kernel does not fit");
    int ctas = nsm * occ;
    if (ctas > kMaxCtas) ctas = kMaxCtas;

    // Time state and species constants (a(t), m(t) as in the context path).
    SetupArgs A;
    std::memset(&A, 0, sizeof(A));
    A.g = g;
    A.ts.t = t;
    A.ts.a = cfg->expansion ? cfg->a0 * std::sqrt(t / cfg->t0) : 1.0;
    if (!(A.ts.a > 0.0)) return report(BEST_ERR_INVALID, "noalloc: a(t) must be positive");
    A.ts.inv_a = 1.0 / A.ts.a;
    A.ts.call = call;
    for (int s = 0; s < S; ++s) {
        const best_species& sp = cfg->species[s];
        MassLaw L{};
        L.m0 = sp.mass0;
        L.m1 = sp.mass1;
        L.n = sp.n_mass_knots;
        for (int k = 0; k < L.n && k < BEST_MAX_MASS_KNOTS; ++k) {
            L.t[k] = sp.mass_t[k];
            L.m[k] = sp.mass_m[k];
        }
        A.ts.mass[s] = mass_at(L, t);
        A.sc[s].stat = cfg->species[s].stat;
        A.sc[s].eta = cfg->species[s].stat == BEST_BE ? 1.0 : (cfg->species[s].stat == BEST_FD ? -1.0 : 0.0);
    }
    A.sd = sd;
    A.td = td;
    A.ctas = ctas;
    const int G = group_size(D, f32);
    A.groups = (td.neval + G - 1) / G;

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    TimeState* ts = reinterpret_cast<TimeState*>(base + kOffTs);
    SpeciesConst* sc = reinterpret_cast<SpeciesConst*>(base + kOffSc);
    SideDesc* dsd = reinterpret_cast<SideDesc*>(base + kOffSide);
    TaskDesc* dtd = reinterpret_cast<TaskDesc*>(base + kOffTask);
    TaskConst* dtc = reinterpret_cast<TaskConst*>(base + kOffTconst);
    SegConst32* dtc32 = reinterpret_cast<SegConst32*>(base + kOffTc32);
    TaskAcc* dacc = reinterpret_cast<TaskAcc*>(base + kOffAcc);
    double* prev = reinterpret_cast<double*>(base + kOffPrev);
    double* knots = reinterpret_cast<double*>(base + kOffKnots);
    float* knots32 = reinterpret_cast<float*>(base + kOffKnots32);
    double* fgrid = reinterpret_cast<double*>(base + kOffFgrid);
    double* coef64 = reinterpret_cast<double*>(base + kOffCoef64);
    float* coef32 = reinterpret_cast<float*>(base + kOffCoef32);

    noalloc_setup_kernel<<<1, 512, 0, st>>>(A, base);
    const size_t spline_smem = 5 * sizeof(double) * n;
    spline_build_kernel<<<S, 256, spline_smem, st>>>(g, f_dev, 0, knots, ts, sc, fgrid, coef64, coef32);
    prepare_kernel<<<1, 32, 0, st>>>(g, dsd, dtd, knots, fgrid, ts, prev, dtc, dacc, 1, nullptr, sc, dtc32);
    float2* map32 = reinterpret_cast<float2*>(base + kOffMap32);
    if (f32) map32_kernel<<<1, 256, 0, st>>>(g, dtd, 1, edges_dev, map32);

    // The sample kernel indexes its descriptor arrays and the map by the
    // segment's task index (0 here: the scratch arrays and the caller's map
    // hold this one task); its Philox stream is keyed by td.gid = task.
    EvalParams P;
    std::memset(&P, 0, sizeof(P));
    P.geo = g;
    P.sides = dsd;
    P.tasks = dtd;
    P.tconst = dtc;
    P.tconst32 = dtc32;
    P.sconst = sc;
    P.ts = ts;
    P.edges = edges_dev;
    P.map32 = map32;
    P.segs = reinterpret_cast<const Segment*>(base + kOffSegs);
    P.cta_seg = reinterpret_cast<const int32_t*>(base + kOffCtaSeg);
    P.n_chunks = ctas;                  // one chunk (segment) per CTA, no counter
    P.chunk_counter = nullptr;
    P.coef = f32 ? static_cast<const void*>(coef32) : static_cast<const void*>(coef64);
    P.knots = f32 ? static_cast<const void*>(knots32) : static_cast<const void*>(knots);
    P.partials = reinterpret_cast<double*>(base + kOffPart);
    P.item_h = nullptr;                 // no stratified sampling here (rejected above)
    P.strat_m = nullptr;
    P.item_rec = nullptr;
    P.itn = iteration;
    P.smem_spline_elems = static_cast<int32_t>(spl);
    const PhiloxKey key = philox_key(g.seed);
    for (int r = 0; r < 20; ++r) P.rk[r] = key.k[r];
    void* args[] = {&P};
    if (cudaLaunchKernel(fn, dim3(ctas), dim3(kThreads), args, smem, st) != cudaSuccess)
        return report(BEST_ERR_CUDA, "noalloc: sample kernel launch failed");
    const int L = 2 + D * nb;
    noalloc_reduce_kernel<<<(L + 255) / 256, 256, 0, st>>>(base, ctas, L, out_dev);
    if (cudaGetLastError() != cudaSuccess) return report(BEST_ERR_CUDA, "noalloc: launch failed");
    return BEST_OK;
}
