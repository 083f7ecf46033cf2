// C ABI of the lbsc library (declared in include/lbsc.h): context life
// cycle, geometry, parameters, stepping (eager launches and CUDA graphs),
// readback, contact angle and checkpoints.
#include "../../include/lbsc.h"
#include "lb_fields.cuh"

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

using namespace lbsc;

namespace lbsc {
int step_occupancy(int precision, int tile_y, bool general, bool tau_one);

}

struct lb_ctx {
    int nx = 0, ny = 0, nz = 0, prec = LB_F32;
    Layout L{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap = nullptr;  // private stream for graph capture
    int device = 0, nsm = 0;
    bool owns = false;
    char* mem = nullptr;
    size_t mem_bytes = 0;
    void* f[2] = {nullptr, nullptr};
    int cur = 0;
    uint32_t* nbmask = nullptr;
    bool general = false;
    int zlo = 0, zhi = 0;
    long long fluid_nodes = 0;
    double* part = nullptr;
    double* red = nullptr;
    double* h_red = nullptr;  // pinned
    Scratch W{};
    lb_params prm{};
    KParams kp{};
    int tile_y = 4, nseg_req = 0;
    int y_tiles_req = 0;  // y-tiles of the step kernel (0 = ceil(ny / tile_y))
    int nseg_cache = 0;  // segments per tile column for the current schedule (0 = not computed)
    long long steps = 0;
    // CUDA graphs of 2^i steps (i = 0 .. kGraphLevels - 1) for each starting buffer
    static constexpr int kGraphLevels = 6;
    cudaGraphExec_t graph[2][kGraphLevels] = {};
    int variant = LB_STEP_AUTO, stages = 0;  // step kernel selection
    CUtensorMap tmap[2][3][4];               // per buffer, per tile height 4/8/16: main box, x strip, y row, corner
    bool tmap_ok[2][3] = {{false, false, false}, {false, false, false}};
    int* dev_err = nullptr;                  // device status word of the step kernels
    uint32_t* clock = nullptr;               // device step counter {steps mod 2^32, done-ticket}
    int halo = 0;                            // z slab: bit 0 plane 0, bit 1 plane nz-1 is a halo plane
    uint32_t hkey = 0;                       // z slab: its planes' offset in the whole lattice (dither key)
    static constexpr int kGraphSteps = 32;
    std::string err;
};

static thread_local std::string g_init_err;

// message for lb_last_error(NULL) from the context-free entry points
void lbsc_set_global_error(const std::string& msg) { g_init_err = msg; }

static int fail(lb_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    else g_init_err = msg;
    return code;
}

static int cuda_fail(lb_ctx* c, cudaError_t e, const char* where)
{
    return fail(c, LB_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LB_CUDA(c, call)                                   \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

static size_t elem_size(int prec) { return prec == LB_F32 ? 4 : 2; }
static size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// rows of nx nodes behind 256 bytes of left padding (x = 0 starts a 256-byte
// unit), at least one node of padding on the right, pitch a multiple of 256
// bytes; one spare row above and below each plane. A warp's paired FP32 access
// to one slot is 256 bytes: aligned to 256 bytes the load-from-global step
// measured 121.2 against 126.1 us at 128^3 (128-byte alignment)
static Layout make_layout(int nx, int ny, int nz, int prec)
{
    Layout L;
    const int line = (int)(256 / (2 * elem_size(prec)));  // nodes (of two values) in 256 bytes
    L.nx = nx;
    L.ny = ny;
    L.nz = nz;
    L.gx = line;
    L.px = (L.gx + nx + 1 + line - 1) / line * line;
    L.plane = (long long)L.px * (ny + 2);
    L.slot = (L.plane * nz + 127) / 128 * 128;
    return L;
}

// memory plan: [f0][f1][nbmask][scratch fields][partials][reduction out]
struct Plan {
    size_t f, mask, scratch, part, red, total;
};
static Plan make_plan(const Layout& L, int prec)
{
    Plan p;
    const long long N = (long long)L.nx * L.ny * L.nz;
    p.f = align256((size_t)2 * Q * L.slot * elem_size(prec));
    p.mask = align256((size_t)L.plane * L.nz * sizeof(uint32_t));
    p.scratch = align256((size_t)10 * N * sizeof(float));
    p.part = align256((size_t)kPartRows * kAngleVals * sizeof(double));
    p.red = align256(64 * sizeof(double));
    p.total = 2 * p.f + p.mask + p.scratch + p.part + p.red;
    return p;
}

// the kernels address a node inside a population slot with a 32-bit offset
static bool dims_ok(int nx, int ny, int nz)
{
    if (nx < 1 || ny < 1 || nz < 1) return false;
    const long long px = ((long long)nx + 64 + 1 + 63) / 64 * 64;
    return px * ((long long)ny + 2) * nz < (1LL << 31) - 256;
}

static FieldArgs field_args(const lb_ctx* c)
{
    FieldArgs F;
    F.L = c->L;
    F.P = c->kp;
    F.general = c->general ? 1 : 0;
    F.nbmask = c->nbmask;
    return F;
}

static void drop_graphs(lb_ctx* c)
{
    c->nseg_cache = 0;
    for (int p = 0; p < 2; ++p)
        for (int i = 0; i < lb_ctx::kGraphLevels; ++i)
            if (c->graph[p][i]) {
                cudaGraphExecDestroy(c->graph[p][i]);
                c->graph[p][i] = nullptr;
            }
}

static void set_kparams(lb_ctx* c)
{
    const lb_params& p = c->prm;
    c->kp.gk = (float)(p.g_br * p.force_scale);
    c->kp.Gax = p.force_weights == LB_WEIGHTS_W36 ? 2.0f : 1.0f;
    c->kp.Gdi = 1.0f;
    c->kp.tau[0] = (float)p.tau_r;
    c->kp.tau[1] = (float)p.tau_b;
    c->kp.itau[0] = (float)(1.0 / p.tau_r);
    c->kp.itau[1] = (float)(1.0 / p.tau_b);
    c->kp.eta[0] = (float)p.eta_wall_r;
    c->kp.eta[1] = (float)p.eta_wall_b;
}

static bool tau_one(const lb_ctx* c) { return c->prm.tau_r == 1.0 && c->prm.tau_b == 1.0; }

static int tma_stages(lb_ctx* c);
static long long tma_call(int op, lb_ctx* c, int ty, int ns);

static int y_tiles(const lb_ctx* c)
{
    return c->y_tiles_req > 0 ? c->y_tiles_req : (c->ny + c->tile_y - 1) / c->tile_y;
}

static int nseg_for(lb_ctx* c, int ncol)
{
    if (c->nseg_cache > 0) return c->nseg_cache;
    const int nzf = c->zhi - c->zlo;
    if (c->nseg_req > 0) return c->nseg_cache = (c->nseg_req < nzf ? c->nseg_req : nzf);
    const int ns = tma_stages(c);
    int occ = ns ? (int)tma_call(2, c, c->tile_y, ns) : step_occupancy(c->prec, c->tile_y, c->general, tau_one(c));
    if (occ < 1) occ = 1;
    const long long target = 2LL * c->nsm * occ;  // about two waves of CTAs
    long long s = (target + ncol - 1) / ncol;
    const long long smax = nzf / 16 > 1 ? nzf / 16 : 1;  // segments of at least 16 planes
    if (s > smax) s = smax;
    if (s < 1) s = 1;
    c->nseg_cache = (int)s;
    return (int)s;
}


// ---------------------------------------------------------------- TMA step support
static const int kTmaTiles[3] = {4, 8, 16};
static int tile_index(int ty) { return ty == 4 ? 0 : (ty == 8 ? 1 : 2); }

template <class S>
static long long tma_op(int op, lb_ctx* c, int ty, int ns, const CUtensorMap* m, const StepArgs<S>* A,
                        cudaStream_t st)
{
    return tma_step<S>(op, ty, ns, tau_one(c), m, A, st);
}

static long long tma_call(int op, lb_ctx* c, int ty, int ns)
{
    switch (c->prec) {
    case LB_F32: return tma_op<float>(op, c, ty, ns, nullptr, nullptr, nullptr);
    case LB_F16: return tma_op<__half>(op, c, ty, ns, nullptr, nullptr, nullptr);
    default: return tma_op<__nv_bfloat16>(op, c, ty, ns, nullptr, nullptr, nullptr);
    }
}

// raise the shared-memory limit of every TMA kernel built for this precision
static cudaError_t tma_prepare(lb_ctx* c)
{
    for (int ty : kTmaTiles)
        for (int ns = 1; ns <= 3; ++ns) {
            const long long e = tma_call(1, c, ty, ns);  // cudaErrorInvalidValue: pair not built
            if (e != (long long)cudaSuccess && e != (long long)cudaErrorInvalidValue) return (cudaError_t)e;
        }
    return cudaSuccess;
}

// stages used by the TMA kernel for the current schedule, 0 if not available
static int tma_stages(lb_ctx* c)
{
    // general geometry always loads from global; AUTO takes the TMA kernel
    // with one stage (measured the faster one for both precisions)
    if (c->general || c->variant == LB_STEP_LDG) return 0;
    const int s0 = c->variant == LB_STEP_AUTO ? 1 : 3, s1 = c->variant == LB_STEP_AUTO ? 1 : 2;
    const int want[2] = {c->stages ? c->stages : s0, c->stages ? c->stages : s1};
    for (int ns : want) {
        // occupancy 0: the pair is not built for this precision (or does not fit)
        const long long occ = tma_call(2, c, c->tile_y, ns);
        if (occ > 0) return ns;
    }
    return 0;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 4-D maps over a population buffer, ordered (x incl. padding, two values per
// node; storage row, spare rows included; plane; slot k). Boxes: main = the
// 32-node tile plus 16 bytes of columns on each side, TY + 2 rows; x strip =
// 16 bytes of columns, TY + 2 rows; y row = the main box's columns, one row;
// corner = 16 bytes of columns, one row. Every box spans one plane and all 19
// slots.
static int tensor_map(lb_ctx* c, int buf, int ty)
{
    const int ti = tile_index(ty);
    if (c->tmap_ok[buf][ti]) return LB_OK;
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(c, LB_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const size_t es = elem_size(c->prec);
    const Layout& L = c->L;
    const cuuint64_t dims[4] = {(cuuint64_t)(2 * L.px), (cuuint64_t)(L.ny + 2), (cuuint64_t)L.nz, (cuuint64_t)Q};
    const cuuint64_t strides[3] = {(cuuint64_t)(2 * L.px) * es, (cuuint64_t)(2 * L.plane) * es,
                                   (cuuint64_t)(2 * L.slot) * es};
    // No L2 promotion: fetching whole 256-byte blocks around the boxes' 16-byte edges raised the
    // step's DRAM reads by a tenth (neighbouring tiles did not reuse the rest in time)
    const cuuint32_t gxv = (cuuint32_t)(16 / es);  // values in 16 bytes
    const cuuint32_t wide = (cuuint32_t)(2 * 32) + 2 * gxv, rows = (cuuint32_t)(ty + 2);
    const cuuint32_t boxes[4][4] = {{wide, rows, 1, (cuuint32_t)Q}, {gxv, rows, 1, (cuuint32_t)Q},
                                    {wide, 1, 1, (cuuint32_t)Q}, {gxv, 1, 1, (cuuint32_t)Q}};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = c->prec == LB_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                   : c->prec == LB_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    for (int kind = 0; kind < 4; ++kind) {
        const CUresult r = enc(&c->tmap[buf][ti][kind], dt, 4, c->f[buf], dims, strides, boxes[kind], estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                               CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(c, LB_ERR_CUDA, "cuTensorMapEncodeTiled failed: " + std::to_string((int)r));
    }
    c->tmap_ok[buf][ti] = true;
    return LB_OK;
}

template <class S>
static StepArgs<S> step_args(lb_ctx* c, int src)
{
    StepArgs<S> A;
    A.src = (const S*)c->f[src];
    A.dst = (S*)c->f[1 - src];
    A.nbmask = c->nbmask;
    A.err = c->dev_err;
    A.clock = c->clock;
    A.L = c->L;
    A.P = c->kp;
    A.tiles_x = (c->nx + 31) / 32;
    A.tiles_y = y_tiles(c);
    A.zlo = c->zlo;
    A.zhi = c->zhi;
    A.nseg = nseg_for(c, A.tiles_x * A.tiles_y);
    A.halo = c->halo;
    A.hkey = c->hkey;
    return A;
}

// one TMA-staged step
template <class S>
static cudaError_t launch_tma(lb_ctx* c, int parity, int ns, cudaStream_t st)
{
    const StepArgs<S> A = step_args<S>(c, parity);
    return (cudaError_t)tma_step<S>(0, c->tile_y, ns, tau_one(c), c->tmap[parity][tile_index(c->tile_y)], &A, st);
}

static cudaError_t launch_steps(lb_ctx* c, int n, int& parity, cudaStream_t st)
{
    const bool t1 = tau_one(c);
    const int ns = tma_stages(c);
    if (ns) {
        for (int b = 0; b < 2; ++b)
            if (tensor_map(c, b, c->tile_y) != LB_OK) return cudaErrorInvalidValue;
    }
    for (int i = 0; i < n; ++i) {
        cudaError_t e;
        if (ns) {
            switch (c->prec) {
            case LB_F32: e = launch_tma<float>(c, parity, ns, st); break;
            case LB_F16: e = launch_tma<__half>(c, parity, ns, st); break;
            default: e = launch_tma<__nv_bfloat16>(c, parity, ns, st); break;
            }
            if (e != cudaSuccess) return e;
            parity ^= 1;
            continue;
        }
        switch (c->prec) {
        case LB_F32: e = launch_step<float>(step_args<float>(c, parity), c->tile_y, c->general, t1, st); break;
        case LB_F16: e = launch_step<__half>(step_args<__half>(c, parity), c->tile_y, c->general, t1, st); break;
        default: e = launch_step<__nv_bfloat16>(step_args<__nv_bfloat16>(c, parity), c->tile_y, c->general, t1, st); break;
        }
        if (e != cudaSuccess) return e;
        parity ^= 1;
    }
    return cudaSuccess;
}

template <class S>
static cudaError_t run_init(lb_ctx* c, const double* drr, const double* drb, int* err = nullptr)
{
    return launch_init<S>(field_args(c), (S*)c->f[0], drr, drb, c->stream, err);
}

static int planar_default(lb_ctx* c)
{
    if (c->nz >= 3) {
        c->general = false;
        c->zlo = 1;
        c->zhi = c->nz - 1;
        c->fluid_nodes = (long long)c->nx * c->ny * (c->nz - 2);
    } else {
        // too thin for walls: fully periodic through an all-fluid mask
        LB_CUDA(c, cudaMemsetAsync(c->nbmask, 0, (size_t)c->L.plane * c->nz * sizeof(uint32_t), c->stream));
        c->general = true;
        c->zlo = 0;
        c->zhi = c->nz;
        c->fluid_nodes = (long long)c->nx * c->ny * c->nz;
    }
    return LB_OK;
}

extern "C" {
static int check_device_status(lb_ctx* c);
}

static int init_common(lb_ctx** out, int nx, int ny, int nz, int precision, const double* rho_r,
                       const double* rho_b, void* stream, void* ext, size_t ext_bytes, int halo = 0, int zbase = 0,
                       const double* ref = nullptr)
{
    if (!out) return fail(nullptr, LB_ERR_ARG, "lb_init: out is NULL");
    *out = nullptr;
    if (!dims_ok(nx, ny, nz)) return fail(nullptr, LB_ERR_ARG, "lb_init: bad lattice dimensions");
    if (precision != LB_F32 && precision != LB_F16 && precision != LB_BF16)
        return fail(nullptr, LB_ERR_ARG, "lb_init: unknown precision");
    if (!rho_r || !rho_b) return fail(nullptr, LB_ERR_ARG, "lb_init: density array is NULL");
    const long long N = (long long)nx * ny * nz;
    for (long long i = 0; i < N; ++i)
        if (!std::isfinite(rho_r[i]) || !std::isfinite(rho_b[i]) || rho_r[i] < 0 || rho_b[i] < 0)
            return fail(nullptr, LB_ERR_ARG, "lb_init: densities must be finite and non-negative");

    lb_ctx* c = new (std::nothrow) lb_ctx();
    if (!c) return fail(nullptr, LB_ERR_CUDA, "lb_init: out of host memory");
    c->nx = nx;
    c->ny = ny;
    c->nz = nz;
    c->prec = precision;
    c->stream = (cudaStream_t)stream;
    c->L = make_layout(nx, ny, nz, precision);
    const Plan p = make_plan(c->L, precision);
    auto bail = [&](int code, const std::string& msg) {
        g_init_err = msg;
        lb_free(c);
        return code;
    };
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bail(LB_ERR_CUDA, std::string("lb_init: ") + cudaGetErrorString(e));
    if (ext) {
        if (ext_bytes < p.total || ((uintptr_t)ext & 255u))
            return bail(LB_ERR_ARG, "lb_init_external: buffer too small or not 256-byte aligned");
        c->mem = (char*)ext;
        c->owns = false;
    } else {
        e = cudaMalloc((void**)&c->mem, p.total);
        if (e != cudaSuccess) return bail(LB_ERR_CUDA, std::string("lb_init: cudaMalloc: ") + cudaGetErrorString(e));
        c->owns = true;
    }
    c->mem_bytes = p.total;
    char* q = c->mem;
    c->f[0] = q;
    q += p.f;
    c->f[1] = q;
    q += p.f;
    c->nbmask = (uint32_t*)q;
    q += p.mask;
    float* sf = (float*)q;
    q += p.scratch;
    c->part = (double*)q;
    q += p.part;
    c->red = (double*)q;
    c->dev_err = (int*)(c->red + 48);
    c->clock = (uint32_t*)(c->red + 50);
    const long long Nn = N;
    c->W.rho[0] = sf + 0 * Nn;
    c->W.rho[1] = sf + 1 * Nn;
    for (int d = 0; d < 3; ++d) c->W.j[d] = sf + (2 + d) * Nn;
    c->W.psi[0] = sf + 5 * Nn;
    c->W.psi[1] = sf + 6 * Nn;
    for (int d = 0; d < 3; ++d) c->W.u[d] = sf + (7 + d) * Nn;
    e = cudaMallocHost((void**)&c->h_red, 64 * sizeof(double));
    if (e != cudaSuccess) return bail(LB_ERR_CUDA, std::string("lb_init: cudaMallocHost: ") + cudaGetErrorString(e));

    if (planar_default(c) != LB_OK) return bail(LB_ERR_CUDA, c->err);
    // reduction area: outputs [0, 32), conservation accumulators [32, 40) and ticket [40], status word, step counter
    e = cudaMemsetAsync(c->red, 0, 64 * sizeof(double), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->dev_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->clock, 0, 2 * sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = tma_prepare(c);
    if (e != cudaSuccess) return bail(LB_ERR_CUDA, std::string("lb_init: ") + cudaGetErrorString(e));
    // 16-bit deviation references: mean initial density over fluid nodes
    double sum[2] = {0, 0};
    long long cnt = 0;
    for (int z = c->zlo; z < c->zhi; ++z)
        for (long long i = (long long)z * nx * ny; i < (long long)(z + 1) * nx * ny; ++i) {
            sum[0] += rho_r[i];
            sum[1] += rho_b[i];
            ++cnt;
        }
    c->kp.ref[0] = precision == LB_F32 ? 0.f : (float)(ref ? ref[0] : sum[0] / (double)cnt);
    c->kp.ref[1] = precision == LB_F32 ? 0.f : (float)(ref ? ref[1] : sum[1] / (double)cnt);
    c->halo = halo;
    c->hkey = (uint32_t)((uint64_t)zbase * (uint64_t)c->L.plane);
    c->prm = lb_params{1.0, 1.0, 0.0, 0.0, 0.0, LB_WEIGHTS_UNIT, 1.0};
    set_kparams(c);

    // stage the densities in the scratch fields (FP64: 2 N doubles fit in 10 N floats)
    double* drr = (double*)sf;
    double* drb = drr + N;
    e = cudaMemcpyAsync(drr, rho_r, N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(drb, rho_b, N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        switch (precision) {
        case LB_F32: e = run_init<float>(c, drr, drb); break;
        case LB_F16: e = run_init<__half>(c, drr, drb); break;
        default: e = run_init<__nv_bfloat16>(c, drr, drb); break;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return bail(LB_ERR_CUDA, std::string("lb_init: ") + cudaGetErrorString(e));
    *out = c;
    return LB_OK;
}

extern "C" {

int lb_init(lb_ctx** out, int nx, int ny, int nz, int precision, const double* rho_r, const double* rho_b,
            void* cuda_stream)
{
    return init_common(out, nx, ny, nz, precision, rho_r, rho_b, cuda_stream, nullptr, 0);
}

int lb_required_bytes(int nx, int ny, int nz, int precision, size_t* bytes)
{
    if (!bytes || !dims_ok(nx, ny, nz)) return fail(nullptr, LB_ERR_ARG, "lb_required_bytes: bad argument");
    if (precision != LB_F32 && precision != LB_F16 && precision != LB_BF16)
        return fail(nullptr, LB_ERR_ARG, "lb_required_bytes: unknown precision");
    *bytes = make_plan(make_layout(nx, ny, nz, precision), precision).total;
    return LB_OK;
}

int lb_init_external(lb_ctx** out, int nx, int ny, int nz, int precision, const double* rho_r,
                     const double* rho_b, void* cuda_stream, void* device_buffer, size_t buffer_bytes)
{
    if (!device_buffer) return fail(nullptr, LB_ERR_ARG, "lb_init_external: device_buffer is NULL");
    return init_common(out, nx, ny, nz, precision, rho_r, rho_b, cuda_stream, device_buffer, buffer_bytes);
}

int lb_init_slab(lb_ctx** out, int nx, int ny, int nz, int precision, const double* rho_r, const double* rho_b,
                 void* cuda_stream, int halo, int zbase, const double* ref)
{
    if (halo < 0 || halo > (LB_HALO_BELOW | LB_HALO_ABOVE))
        return fail(nullptr, LB_ERR_ARG, "lb_init_slab: halo must be a combination of LB_HALO_BELOW and LB_HALO_ABOVE");
    if (nz < 3 || zbase < 0) return fail(nullptr, LB_ERR_ARG, "lb_init_slab: a slab needs nz >= 3 and zbase >= 0");
    // the boundary plane a slab sends must be final after its own step: with neighbours on both faces, a
    // single owned plane would receive its crossing populations from one face only after sending to the other
    if (halo == (LB_HALO_BELOW | LB_HALO_ABOVE) && nz < 4)
        return fail(nullptr, LB_ERR_ARG, "lb_init_slab: a slab with neighbours on both faces needs two owned planes");
    if (ref && !(std::isfinite(ref[0]) && std::isfinite(ref[1])))
        return fail(nullptr, LB_ERR_ARG, "lb_init_slab: reference densities must be finite");
    return init_common(out, nx, ny, nz, precision, rho_r, rho_b, cuda_stream, nullptr, 0, halo, zbase, ref);
}

int lb_halo_bytes(lb_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(c, LB_ERR_ARG, "lb_halo_bytes: NULL argument");
    *bytes = (size_t)kHaloEntries * c->nx * c->ny * elem_size(c->prec);
    return LB_OK;
}

static int halo_copy(lb_ctx* c, int face, void* msg, int unpack, const char* who)
{
    if (!c || !msg || (face != 0 && face != 1)) return fail(c, LB_ERR_ARG, std::string(who) + ": bad argument");
    if (!(c->halo & (1 << face))) return fail(c, LB_ERR_STATE, std::string(who) + ": no halo plane on that face");
    LB_CUDA(c, launch_halo_copy(c->L, c->f[c->cur], elem_size(c->prec), msg, face, unpack, c->stream));
    return LB_OK;
}

int lb_halo_pack(lb_ctx* c, int face, void* msg) { return halo_copy(c, face, msg, 0, "lb_halo_pack"); }

int lb_halo_unpack(lb_ctx* c, int face, const void* msg)
{
    return halo_copy(c, face, const_cast<void*>(msg), 1, "lb_halo_unpack");
}

static bool slab_pair_ok(const lb_ctx* a, const lb_ctx* b)
{
    return a && b && a != b && a->nx == b->nx && a->ny == b->ny && a->prec == b->prec && a->L.px == b->L.px &&
           (a->halo & LB_HALO_ABOVE) && (b->halo & LB_HALO_BELOW);
}

int lb_halo_exchange(lb_ctx* below, lb_ctx* above)
{
    if (!slab_pair_ok(below, above))
        return fail(below, LB_ERR_ARG, "lb_halo_exchange: need a slab with a halo above and one with a halo below, "
                                       "same nx, ny and precision");
    if (below->stream != above->stream)
        return fail(below, LB_ERR_ARG, "lb_halo_exchange: the two slabs must share one stream");
    LB_CUDA(below, launch_halo_exchange(below->L, below->f[below->cur], above->L, above->f[above->cur],
                                        elem_size(below->prec), below->stream));
    return LB_OK;
}

int lb_slabs_step(lb_ctx* const* slabs, int nslab, int nsteps)
{
    if (!slabs || nslab < 1 || nsteps < 0) return fail(nullptr, LB_ERR_ARG, "lb_slabs_step: bad argument");
    for (int i = 0; i < nslab; ++i) {
        if (!slabs[i]) return fail(nullptr, LB_ERR_ARG, "lb_slabs_step: NULL slab");
        const int want = (i > 0 ? LB_HALO_BELOW : 0) | (i + 1 < nslab ? LB_HALO_ABOVE : 0);
        if (slabs[i]->halo != want || slabs[i]->stream != slabs[0]->stream)
            return fail(slabs[i], LB_ERR_ARG, "lb_slabs_step: slabs must be ordered bottom to top, with halo planes "
                                              "exactly on their inner faces, on one stream");
        if (i > 0 && !slab_pair_ok(slabs[i - 1], slabs[i]))
            return fail(slabs[i], LB_ERR_ARG, "lb_slabs_step: neighbouring slabs differ in nx, ny or precision");
    }
    for (int t = 0; t < nsteps; ++t) {
        for (int i = 0; i < nslab; ++i) {
            const int rc = lb_step(slabs[i], 1);
            if (rc != LB_OK) return rc;
        }
        for (int i = 0; i + 1 < nslab; ++i) {
            const int rc = lb_halo_exchange(slabs[i], slabs[i + 1]);
            if (rc != LB_OK) return rc;
        }
    }
    return LB_OK;
}

int lb_reset(lb_ctx* c, const double* rho_r, const double* rho_b)
{
    if (!c || !rho_r || !rho_b) return fail(c, LB_ERR_ARG, "lb_reset: NULL argument");
    const long long N = (long long)c->nx * c->ny * c->nz;
    // stage the densities in the scratch fields (FP64: 2 N doubles fit in 10 N floats)
    double* drr = (double*)c->W.rho[0];
    double* drb = drr + N;
    LB_CUDA(c, cudaMemcpyAsync(drr, rho_r, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, cudaMemcpyAsync(drb, rho_b, N * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    cudaError_t e;
    switch (c->prec) {
    case LB_F32: e = run_init<float>(c, drr, drb, c->dev_err); break;
    case LB_F16: e = run_init<__half>(c, drr, drb, c->dev_err); break;
    default: e = run_init<__nv_bfloat16>(c, drr, drb, c->dev_err); break;
    }
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_reset: init");
    LB_CUDA(c, launch_clock_set(c->clock, 0, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->cur = 0;
    c->steps = 0;
    int h = 0;
    LB_CUDA(c, cudaMemcpy(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & kErrInput) {
        LB_CUDA(c, cudaMemset(c->dev_err, 0, sizeof(int)));
        return fail(c, LB_ERR_ARG, "lb_reset: densities must be finite and non-negative");
    }
    return check_device_status(c);
}

int lb_set_geometry(lb_ctx* c, const uint8_t* solid)
{
    if (!c || !solid) return fail(c, LB_ERR_ARG, "lb_set_geometry: NULL argument");
    if (c->halo) return fail(c, LB_ERR_UNSUPPORTED, "lb_set_geometry: a z slab keeps the planar walls");
    const int nx = c->nx, ny = c->ny, nz = c->nz;
    const long long N = (long long)nx * ny * nz, NP = (long long)nx * ny;
    long long fluid = 0;
    bool planar = nz >= 3;
    for (long long i = 0; i < N; ++i) {
        const bool s = solid[i] != 0;
        fluid += !s;
        const long long z = i / NP;
        if (s != (z == 0 || z == nz - 1)) planar = false;
    }
    if (fluid == 0) return fail(c, LB_ERR_ARG, "lb_set_geometry: no fluid node");
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    drop_graphs(c);
    c->fluid_nodes = fluid;
    if (planar) {
        c->general = false;
        c->zlo = 1;
        c->zhi = nz - 1;
        return LB_OK;
    }
    std::vector<uint32_t> m((size_t)c->L.plane * nz, 0u);
    auto at = [&](int x, int y, int z) { return solid[(long long)x + (long long)nx * (y + (long long)ny * z)] != 0; };
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                uint32_t b = at(x, y, z) ? kSelfSolid : 0u;
                for (int k = 1; k < Q; ++k)
                    if (at(wrapi(x + cx(k), nx), wrapi(y + cy(k), ny), wrapi(z + cz(k), nz))) b |= 1u << k;
                m[(size_t)c->L.off(x, y, z)] = b;
            }
    LB_CUDA(c, cudaMemcpy(c->nbmask, m.data(), m.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
    c->general = true;
    c->zlo = 0;
    c->zhi = nz;
    return LB_OK;
}

int lb_set_params(lb_ctx* c, const lb_params* p)
{
    if (!c || !p) return fail(c, LB_ERR_ARG, "lb_set_params: NULL argument");
    const double v[] = {p->tau_r, p->tau_b, p->g_br, p->eta_wall_r, p->eta_wall_b, p->force_scale};
    for (double x : v)
        if (!std::isfinite(x)) return fail(c, LB_ERR_ARG, "lb_set_params: non-finite value");
    if (p->tau_r <= 0.5 || p->tau_b <= 0.5) return fail(c, LB_ERR_ARG, "lb_set_params: tau must exceed 1/2");
    if (p->force_weights != LB_WEIGHTS_UNIT && p->force_weights != LB_WEIGHTS_W36)
        return fail(c, LB_ERR_ARG, "lb_set_params: unknown force_weights");
    drop_graphs(c);
    c->prm = *p;
    set_kparams(c);
    return LB_OK;
}

int lb_build_flags(int* flags)
{
    if (!flags) return LB_ERR_ARG;
    *flags = kCheckBounds ? LB_BUILD_BOUNDS_CHECKED : 0;
    return LB_OK;
}

int lb_selftest_bounded_wait(lb_ctx* c, unsigned spin_limit)
{
    if (!c || spin_limit < 1 || spin_limit > (1u << 20))
        return fail(c, LB_ERR_ARG, "lb_selftest_bounded_wait: spin_limit in [1, 2^20]");
    LB_CUDA(c, launch_wait_probe(c->dev_err, spin_limit, c->stream));
    return lb_sync(c);
}

int lb_set_step_variant(lb_ctx* c, int variant, int stages)
{
    if (!c) return fail(c, LB_ERR_ARG, "lb_set_step_variant: NULL context");
    if (variant < LB_STEP_AUTO || variant > LB_STEP_TMA || stages < 0 || stages > 3)
        return fail(c, LB_ERR_ARG, "lb_set_step_variant: unknown variant or stages");
    drop_graphs(c);
    c->variant = variant;
    c->stages = stages;
    return LB_OK;
}

int lb_set_tiling(lb_ctx* c, int tile_y, int y_tiles, int z_segments)
{
    if (!c) return fail(c, LB_ERR_ARG, "lb_set_tiling: NULL context");
    if ((tile_y != 4 && tile_y != 8 && tile_y != 16) || z_segments < 0)
        return fail(c, LB_ERR_ARG, "lb_set_tiling: tile_y must be 4, 8 or 16 and z_segments >= 0");
    if (y_tiles < 0 || y_tiles > c->ny || (y_tiles > 0 && (c->ny + y_tiles - 1) / y_tiles > tile_y))
        return fail(c, LB_ERR_ARG, "lb_set_tiling: y_tiles must be 0 or split ny into rows of at most tile_y");
    if (y_tiles > 0 && (long long)((c->nx + 31) / 32) * y_tiles * (z_segments > 0 ? z_segments : 1) > (1LL << 30))
        return fail(c, LB_ERR_ARG, "lb_set_tiling: too many tiles");
    drop_graphs(c);
    c->tile_y = tile_y;
    c->y_tiles_req = y_tiles;
    c->nseg_req = z_segments;
    return LB_OK;
}

int lb_set_schedule(lb_ctx* c, int tile_y, int z_segments)
{
    if (!c) return fail(c, LB_ERR_ARG, "lb_set_schedule: NULL context");
    return lb_set_tiling(c, tile_y, 0, z_segments);
}

// Capture the step graphs of every size for both starting buffers (after a
// change of schedule or parameters dropped them), so that no later call
// captures inside a caller's timed or captured region.
static int capture_graphs(lb_ctx* c)
{
    if (c->graph[0][0]) return LB_OK;
    nseg_for(c, ((c->nx + 31) / 32) * y_tiles(c));
    for (int p = 0; p < 2; ++p)
        for (int i = 0; i < lb_ctx::kGraphLevels; ++i) {
            cudaGraph_t g = nullptr;
            LB_CUDA(c, cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
            int p2 = p;
            cudaError_t e = launch_steps(c, 1 << i, p2, c->cap);
            cudaError_t e2 = cudaStreamEndCapture(c->cap, &g);
            if (e != cudaSuccess) return cuda_fail(c, e, "lb_step: capture");
            if (e2 != cudaSuccess) return cuda_fail(c, e2, "lb_step: end capture");
            e = cudaGraphInstantiate(&c->graph[p][i], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(c, e, "lb_step: graph instantiate");
        }
    return LB_OK;
}

int lb_step(lb_ctx* c, int nsteps)
{
    if (!c || nsteps < 0) return fail(c, LB_ERR_ARG, "lb_step: bad argument");
    if (nsteps == 0) return LB_OK;
    const int ns = tma_stages(c);
    // n steps as graphs of 2^i steps: one launch per set bit (and per 32 steps),
    // so that consecutive kernels follow each other without host launch gaps
    const int rc = capture_graphs(c);
    if (rc != LB_OK) return rc;
    constexpr int top = lb_ctx::kGraphLevels - 1;
    int par = c->cur, n = nsteps;
    while (n >= (1 << top)) {
        LB_CUDA(c, cudaGraphLaunch(c->graph[par][top], c->stream));
        n -= 1 << top;  // an even number of steps: the buffers end where they began
    }
    for (int i = top - 1; i >= 0; --i)
        if (n & (1 << i)) {
            LB_CUDA(c, cudaGraphLaunch(c->graph[par][i], c->stream));
            if (i == 0) par ^= 1;
        }
    c->cur = par;
    c->steps += nsteps;
    return LB_OK;
}

int lb_sync(lb_ctx* c)
{
    if (!c) return fail(c, LB_ERR_ARG, "lb_sync: NULL context");
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    LB_CUDA(c, cudaGetLastError());
    return check_device_status(c);
}

}  // extern "C"

template <class S>
static cudaError_t run_cons(lb_ctx* c, float* phi)
{
    return launch_conservation<S>(field_args(c), (const S*)c->f[c->cur], (unsigned long long*)(c->red + 32),
                                  (unsigned int*)(c->red + 40), c->red, c->stream, phi);
}
template <class S>
static cudaError_t run_fields(lb_ctx* c, bool vel)
{
    return launch_fields<S>(field_args(c), (const S*)c->f[c->cur], c->W, vel, c->stream);
}

static cudaError_t dispatch_cons(lb_ctx* c, float* phi = nullptr)
{
    switch (c->prec) {
    case LB_F32: return run_cons<float>(c, phi);
    case LB_F16: return run_cons<__half>(c, phi);
    default: return run_cons<__nv_bfloat16>(c, phi);
    }
}
template <class S>
static cudaError_t run_phi(lb_ctx* c)
{
    return launch_phi<S>(field_args(c), (const S*)c->f[c->cur], c->W, c->stream);
}
static cudaError_t dispatch_phi(lb_ctx* c)
{
    switch (c->prec) {
    case LB_F32: return run_phi<float>(c);
    case LB_F16: return run_phi<__half>(c);
    default: return run_phi<__nv_bfloat16>(c);
    }
}
static cudaError_t dispatch_fields(lb_ctx* c, bool vel)
{
    switch (c->prec) {
    case LB_F32: return run_fields<float>(c, vel);
    case LB_F16: return run_fields<__half>(c, vel);
    default: return run_fields<__nv_bfloat16>(c, vel);
    }
}

extern "C" {

// the conservation sums (and, with phi, the contact angle's phi field) of the
// current state into cons[8]
static int conservation_impl(lb_ctx* c, double cons[8], float* phi)
{
    LB_CUDA(c, dispatch_cons(c, phi));
    LB_CUDA(c, cudaMemcpyAsync(c->h_red, c->red, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 7; ++i) cons[i] = c->h_red[i];
    cons[7] = (double)c->steps;
    const int st = check_device_status(c);
    if (st != LB_OK) return st;
    if (cons[5] > 0) return fail(c, LB_ERR_NAN, "non-finite populations in the state");
    return LB_OK;
}

int lb_conservation(lb_ctx* c, double cons[8])
{
    if (!c || !cons) return fail(c, LB_ERR_ARG, "lb_conservation: NULL argument");
    return conservation_impl(c, cons, nullptr);
}

int lb_moments(lb_ctx* c, double* rho_r, double* rho_b, double* u, double cons[8])
{
    if (!c) return fail(c, LB_ERR_ARG, "lb_moments: NULL context");
    const long long N = (long long)c->nx * c->ny * c->nz;
    if (rho_r || rho_b || u) {
        LB_CUDA(c, dispatch_fields(c, u != nullptr));
        std::vector<float> tmp((size_t)N);
        auto pull = [&](const float* src, double* dst) -> int {
            LB_CUDA(c, cudaMemcpyAsync(tmp.data(), src, N * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
            LB_CUDA(c, cudaStreamSynchronize(c->stream));
            for (long long i = 0; i < N; ++i) dst[i] = tmp[i];
            return LB_OK;
        };
        int rc;
        if (rho_r && (rc = pull(c->W.rho[0], rho_r)) != LB_OK) return rc;
        if (rho_b && (rc = pull(c->W.rho[1], rho_b)) != LB_OK) return rc;
        if (u)
            for (int d = 0; d < 3; ++d)
                if ((rc = pull(c->W.u[d], u + d * N)) != LB_OK) return rc;
    }
    double tmp[8];
    int rc = lb_conservation(c, tmp);
    if (cons) memcpy(cons, tmp, sizeof(tmp));
    return rc;
}

static int solve4(double M[4][4], double v[4], double s[4])
{
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (std::fabs(M[r][col]) > std::fabs(M[piv][col])) piv = r;
        if (std::fabs(M[piv][col]) < 1e-300) return -1;
        if (piv != col) {
            for (int k = 0; k < 4; ++k) std::swap(M[col][k], M[piv][k]);
            std::swap(v[col], v[piv]);
        }
        for (int r = col + 1; r < 4; ++r) {
            const double f = M[r][col] / M[col][col];
            for (int k = col; k < 4; ++k) M[r][k] -= f * M[col][k];
            v[r] -= f * v[col];
        }
    }
    for (int r = 3; r >= 0; --r) {
        double a = v[r];
        for (int k = r + 1; k < 4; ++k) a -= M[r][k] * s[k];
        s[r] = a / M[r][r];
    }
    return 0;
}

// the droplet of the phi field in c->W (written by the phi pass or the
// conservation pass of the current state)
static int angle_from_phi(lb_ctx* c, double offset, double level, lb_droplet* out);

int lb_contact_angle(lb_ctx* c, double offset, lb_droplet* out) { return lb_contact_angle_at(c, offset, 0.0, out); }

int lb_contact_angle_at(lb_ctx* c, double offset, double level, lb_droplet* out)
{
    if (!c || !out || !(offset >= 0) || !std::isfinite(offset) || !std::isfinite(level))
        return fail(c, LB_ERR_ARG, "lb_contact_angle: bad argument");
    LB_CUDA(c, dispatch_phi(c));
    return angle_from_phi(c, offset, level, out);
}

int lb_measure(lb_ctx* c, double cons[8], double offset, lb_droplet* out)
{
    if (!c || !cons || !out || !(offset >= 0) || !std::isfinite(offset))
        return fail(c, LB_ERR_ARG, "lb_measure: bad argument");
    const int rc = conservation_impl(c, cons, c->W.rho[0]);
    if (rc != LB_OK) return rc;
    return angle_from_phi(c, offset, 0.0, out);
}

static int angle_from_phi(lb_ctx* c, double offset, double level, lb_droplet* out)
{
    memset(out, 0, sizeof(*out));
    const double zw = 0.5, zref = zw + offset;
    LB_CUDA(c, launch_angle(field_args(c), c->W, zref, level, c->part, c->red, c->stream));
    LB_CUDA(c, cudaMemcpyAsync(c->h_red, c->red, kAngleVals * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    const double* v = c->h_red;
    const double top = v[0], area = v[1];
    const int npts = (int)v[2];
    const double h = top - zw;
    const double pi = 3.14159265358979323846;
    const double bref = 2.0 * std::sqrt(area / pi), hp = h - offset;
    out->h = h;
    out->base_ref = bref;
    out->phi_max = v[17];
    out->phi_min = -v[18];
    const int z0 = (int)std::floor(zref);
    if (!(z0 >= 0 && z0 + 1 < c->nz)) out->status = LB_DROP_BAD_PLANE;
    else if (!(v[17] > -1e299) || !((double)v[17] - level > 0)) out->status = LB_DROP_NO_PHASE;
    else if (!(top > -1e299)) out->status = LB_DROP_NO_APEX;
    else if (!(hp > 0)) out->status = LB_DROP_LOW_APEX;
    else if (!(bref > 0)) out->status = LB_DROP_NO_BASE;
    else out->status = LB_DROP_OK;
    if (out->status == LB_DROP_OK) {
        // cap above the reference plane: height hp, base bref -> sphere radius (Fig. 2 relation)
        const double r = (0.25 * bref * bref + hp * hp) / (2.0 * hp);
        const double arg = r * r - (r - h) * (r - h);
        const double b = 2.0 * std::sqrt(arg > 0 ? arg : 0.0);
        out->r = r;
        out->b = b;
        out->theta_deg = std::atan2(0.5 * b, r - h) * 180.0 / pi;
        out->ok = 1;
    }
    out->n_points = npts;
    if (npts >= 4) {
        double M[4][4], rhs[4], s[4];
        int m = 3;
        for (int r = 0; r < 4; ++r)
            for (int q = r; q < 4; ++q) M[r][q] = M[q][r] = v[m++];
        for (int r = 0; r < 4; ++r) rhs[r] = v[13 + r];
        if (solve4(M, rhs, s) == 0) {
            const double R2 = s[3] + s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
            if (R2 > 0) {
                const double R = std::sqrt(R2);
                double cth = -(s[2] - zw) / R;
                cth = cth > 1 ? 1 : (cth < -1 ? -1 : cth);
                out->xc = s[0];
                out->yc = s[1];
                out->zc = s[2];
                out->r_fit = R;
                out->theta_fit_deg = std::acos(cth) * 180.0 / pi;
            }
        }
    }
    return LB_OK;
}

// Read and clear the step kernels' device status word (the stream is idle).
static int check_device_status(lb_ctx* c)
{
    int h = 0;
    LB_CUDA(c, cudaMemcpy(&h, c->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        LB_CUDA(c, cudaMemset(c->dev_err, 0, sizeof(int)));
        if (h & kErrBounds)
            return fail(c, LB_ERR_STATE, "an index fell outside its buffer (bounds-checked build); the access was skipped");
        return fail(c, LB_ERR_BARRIER_TIMEOUT, "a bounded wait in the step kernel gave up (TMA stage never landed)");
    }
    return LB_OK;
}

struct StateHeader {
    char magic[8];
    int nx, ny, nz, prec;
    long long steps;
    long long payload;
};

static size_t payload_bytes(const lb_ctx* c) { return (size_t)2 * Q * c->L.slot * elem_size(c->prec); }

int lb_state_bytes(lb_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return fail(c, LB_ERR_ARG, "lb_state_bytes: NULL argument");
    *bytes = sizeof(StateHeader) + payload_bytes(c);
    return LB_OK;
}

int lb_save(lb_ctx* c, void* host, size_t bytes)
{
    if (!c || !host) return fail(c, LB_ERR_ARG, "lb_save: NULL argument");
    const size_t pb = payload_bytes(c);
    if (bytes < sizeof(StateHeader) + pb) return fail(c, LB_ERR_ARG, "lb_save: buffer too small");
    StateHeader h;
    memcpy(h.magic, "LBSCST02", 8);
    h.nx = c->nx;
    h.ny = c->ny;
    h.nz = c->nz;
    h.prec = c->prec;
    h.steps = c->steps;
    h.payload = (long long)pb;
    memcpy(host, &h, sizeof(h));
    LB_CUDA(c, cudaMemcpyAsync((char*)host + sizeof(h), c->f[c->cur], pb, cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    return LB_OK;
}

int lb_load(lb_ctx* c, const void* host, size_t bytes)
{
    if (!c || !host) return fail(c, LB_ERR_ARG, "lb_load: NULL argument");
    const size_t pb = payload_bytes(c);
    if (bytes < sizeof(StateHeader)) return fail(c, LB_ERR_ARG, "lb_load: truncated state");
    StateHeader h;
    memcpy(&h, host, sizeof(h));
    if (memcmp(h.magic, "LBSCST02", 8) != 0) return fail(c, LB_ERR_ARG, "lb_load: not an lbsc state");
    if (h.nx != c->nx || h.ny != c->ny || h.nz != c->nz || h.prec != c->prec || h.payload != (long long)pb)
        return fail(c, LB_ERR_ARG, "lb_load: state does not match this context");
    if (bytes < sizeof(StateHeader) + pb) return fail(c, LB_ERR_ARG, "lb_load: truncated state");
    LB_CUDA(c, cudaMemcpyAsync(c->f[c->cur], (const char*)host + sizeof(h), pb, cudaMemcpyHostToDevice, c->stream));
    LB_CUDA(c, launch_clock_set(c->clock, (uint32_t)h.steps, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    c->steps = h.steps;
    return LB_OK;
}

}  // extern "C"

template <class S>
static cudaError_t run_get(lb_ctx* c, double* d)
{
    return launch_get_pop<S>(field_args(c), (const S*)c->f[c->cur], d, c->stream);
}
template <class S>
static cudaError_t run_set(lb_ctx* c, const double* d)
{
    return launch_set_pop<S>(field_args(c), (S*)c->f[c->cur], d, c->stream);
}

extern "C" {

int lb_get_populations(lb_ctx* c, double* n)
{
    if (!c || !n) return fail(c, LB_ERR_ARG, "lb_get_populations: NULL argument");
    const size_t bytes = (size_t)2 * Q * c->nx * c->ny * c->nz * sizeof(double);
    double* d = nullptr;
    LB_CUDA(c, cudaMalloc((void**)&d, bytes));
    cudaError_t e;
    switch (c->prec) {
    case LB_F32: e = run_get<float>(c, d); break;
    case LB_F16: e = run_get<__half>(c, d); break;
    default: e = run_get<__nv_bfloat16>(c, d); break;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(n, d, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_get_populations");
    return LB_OK;
}

int lb_set_populations(lb_ctx* c, const double* n)
{
    if (!c || !n) return fail(c, LB_ERR_ARG, "lb_set_populations: NULL argument");
    const size_t bytes = (size_t)2 * Q * c->nx * c->ny * c->nz * sizeof(double);
    double* d = nullptr;
    LB_CUDA(c, cudaMalloc((void**)&d, bytes));
    cudaError_t e = cudaMemcpyAsync(d, n, bytes, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) {
        switch (c->prec) {
        case LB_F32: e = run_set<float>(c, d); break;
        case LB_F16: e = run_set<__half>(c, d); break;
        default: e = run_set<__nv_bfloat16>(c, d); break;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(c, e, "lb_set_populations");
    return LB_OK;
}

const char* lb_last_error(const lb_ctx* c)
{
    if (!c) return g_init_err.c_str();
    return c->err.c_str();
}

void lb_free(lb_ctx* c)
{
    if (!c) return;
    if (c->stream || c->mem) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->owns && c->mem) cudaFree(c->mem);
    if (c->h_red) cudaFreeHost(c->h_red);
    if (c->cap) cudaStreamDestroy(c->cap);
    delete c;
}

}  // extern "C"

// ====================================================================== batch
// Many independent lattices (their own sizes and parameters) advanced by one
// persistent kernel launch per step over a shared work list. Each box is a
// full context living in a slice of one device allocation, so every per-box
// readback (moments, contact angle, checkpoints) is the single-lattice code.

struct lb_batch {
    int nbox = 0, prec = LB_F32;
    cudaStream_t stream = nullptr, cap = nullptr;
    std::vector<lb_ctx*> box;
    char* mem = nullptr;
    void* dargs = nullptr;  // StepArgs<S>[2*nbox]: box i read from buffer parity p at 2*i + p
    uint32_t* done = nullptr; // CTAs finished in the current step (the last one advances the boxes' counters)
    int4* ditems = nullptr; // (box, tile column, first plane, end plane)
    void* dmaps = nullptr;  // TMA variant: the four tensor maps of box i, source buffer p, at 2*i + p
    int nitems = 0;
    int tile_y = 8, seg_planes = 32, ctas_per_sm = 0, grid = 0;
    int variant = LB_STEP_AUTO;
    bool tma = false;       // the TMA-staged batch kernel runs the steps
    bool tau1 = true;
    int cur = 0;
    long long steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    std::string err;
};

static int bfail(lb_batch* b, int code, const std::string& msg)
{
    if (b) b->err = msg;
    else g_init_err = msg;
    return code;
}

#define LB_BCUDA(b, call)                                                                           \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

static void batch_drop_graphs(lb_batch* b)
{
    for (int i = 0; i < 2; ++i)
        if (b->graph[i]) {
            cudaGraphExecDestroy(b->graph[i]);
            b->graph[i] = nullptr;
        }
}

template <class S>
static int batch_build_typed(lb_batch* b)
{
    std::vector<StepArgs<S>> args(2 * (size_t)b->nbox);
    std::vector<int4> items;
    b->tau1 = true;
    for (int i = 0; i < b->nbox; ++i) {
        lb_ctx* c = b->box[i];
        c->tile_y = b->tile_y;
        b->tau1 = b->tau1 && tau_one(c);
        for (int p = 0; p < 2; ++p) args[2 * i + p] = step_args<S>(c, p);
        const int tx = (c->nx + 31) / 32, ty = (c->ny + b->tile_y - 1) / b->tile_y;
        const int nzf = c->zhi - c->zlo;
        int nseg = (nzf + b->seg_planes / 2) / b->seg_planes;
        nseg = nseg < 1 ? 1 : (nseg > nzf ? nzf : nseg);
        for (int s = 0; s < nseg; ++s) {
            const int za = c->zlo + (int)((long long)s * nzf / nseg), zb = c->zlo + (int)((long long)(s + 1) * nzf / nseg);
            if (za >= zb) continue;
            for (int col = 0; col < tx * ty; ++col) items.push_back(make_int4(i, col, za, zb));
        }
    }
    if (b->dargs) cudaFree(b->dargs);
    if (b->ditems) cudaFree(b->ditems);
    if (b->dmaps) cudaFree(b->dmaps);
    b->dargs = nullptr;
    b->ditems = nullptr;
    b->dmaps = nullptr;
    const size_t abytes = align256(args.size() * sizeof(StepArgs<S>));
    LB_BCUDA(b, cudaMalloc(&b->dargs, abytes + 256));
    b->done = (uint32_t*)((char*)b->dargs + abytes);
    LB_BCUDA(b, cudaMemset(b->done, 0, sizeof(uint32_t)));
    LB_BCUDA(b, cudaMalloc((void**)&b->ditems, items.size() * sizeof(int4)));
    LB_BCUDA(b, cudaMemcpy(b->dargs, args.data(), args.size() * sizeof(StepArgs<S>), cudaMemcpyHostToDevice));
    LB_BCUDA(b, cudaMemcpy(b->ditems, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice));
    b->nitems = (int)items.size();
    // AUTO and TMA take the TMA-staged batch kernel where it is built (one
    // stage, 4- or 8-row tiles); LDG the load-from-global one
    // (the shared-memory attribute first: the occupancy of a kernel above 48 KB counts 0 without it)
    b->tma = b->variant != LB_STEP_LDG &&
             tma_batch<S>(1, b->tile_y, b->tau1, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, 0, nullptr) ==
                 (long long)cudaSuccess &&
             tma_batch<S>(2, b->tile_y, b->tau1, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, 0, nullptr) > 0;
    if (b->tma) {
        std::vector<CUtensorMap> maps(8 * (size_t)b->nbox);
        for (int i = 0; i < b->nbox; ++i) {
            lb_ctx* c = b->box[i];
            for (int p = 0; p < 2; ++p) {
                const int rc = tensor_map(c, p, b->tile_y);
                if (rc != LB_OK) return bfail(b, rc, c->err);
                for (int k = 0; k < 4; ++k) maps[8 * i + 4 * p + k] = c->tmap[p][tile_index(b->tile_y)][k];
            }
        }
        LB_BCUDA(b, cudaMalloc(&b->dmaps, maps.size() * sizeof(CUtensorMap)));  // 256-byte aligned
        LB_BCUDA(b, cudaMemcpy(b->dmaps, maps.data(), maps.size() * sizeof(CUtensorMap), cudaMemcpyHostToDevice));
    }
    const int occ = b->ctas_per_sm > 0
                        ? b->ctas_per_sm
                        : (b->tma ? (int)tma_batch<S>(2, b->tile_y, b->tau1, nullptr, nullptr, nullptr, 0, 0, 0,
                                                      nullptr, 0, nullptr)
                                  : batch_occupancy<S>(b->tile_y, b->tau1));
    b->grid = b->box[0]->nsm * (occ > 0 ? occ : 1);
    return LB_OK;
}

static int batch_build(lb_batch* b)
{
    batch_drop_graphs(b);
    switch (b->prec) {
    case LB_F32: return batch_build_typed<float>(b);
    case LB_F16: return batch_build_typed<__half>(b);
    default: return batch_build_typed<__nv_bfloat16>(b);
    }
}

template <class S>
static cudaError_t batch_launch_tma(lb_batch* b, int parity, cudaStream_t st)
{
    return (cudaError_t)tma_batch<S>(0, b->tile_y, b->tau1, b->dmaps, (const StepArgs<S>*)b->dargs, b->ditems,
                                     b->nitems, parity, b->nbox, b->done, b->grid, st);
}

static cudaError_t batch_launch(lb_batch* b, int parity, cudaStream_t st)
{
    if (b->tma) {
        switch (b->prec) {
        case LB_F32: return batch_launch_tma<float>(b, parity, st);
        case LB_F16: return batch_launch_tma<__half>(b, parity, st);
        default: return batch_launch_tma<__nv_bfloat16>(b, parity, st);
        }
    }
    switch (b->prec) {
    case LB_F32:
        return launch_batch_step<float>((const StepArgs<float>*)b->dargs, b->ditems, b->nitems, parity, b->tile_y,
                                        b->tau1, b->grid, b->nbox, b->done, st);
    case LB_F16:
        return launch_batch_step<__half>((const StepArgs<__half>*)b->dargs, b->ditems, b->nitems, parity, b->tile_y,
                                         b->tau1, b->grid, b->nbox, b->done, st);
    default:
        return launch_batch_step<__nv_bfloat16>((const StepArgs<__nv_bfloat16>*)b->dargs, b->ditems, b->nitems, parity,
                                                b->tile_y, b->tau1, b->grid, b->nbox, b->done, st);
    }
}

extern "C" {

int lb_batch_create(lb_batch** out, int nbox, const int* dims, const double* rho_r, const double* rho_b,
                    const lb_params* params, int precision, void* cuda_stream)
{
    if (!out) return bfail(nullptr, LB_ERR_ARG, "lb_batch_create: out is NULL");
    *out = nullptr;
    if (nbox < 1 || !dims || !rho_r || !rho_b || !params) return bfail(nullptr, LB_ERR_ARG, "lb_batch_create: bad argument");
    if (precision != LB_F32 && precision != LB_F16 && precision != LB_BF16)
        return bfail(nullptr, LB_ERR_ARG, "lb_batch_create: unknown precision");
    std::vector<size_t> off(nbox);
    size_t total = 0;
    for (int i = 0; i < nbox; ++i) {
        const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        if (!dims_ok(nx, ny, nz) || nz < 3) return bfail(nullptr, LB_ERR_ARG, "lb_batch_create: bad box dimensions");
        off[i] = total;
        total += align256(make_plan(make_layout(nx, ny, nz, precision), precision).total);
    }
    lb_batch* b = new (std::nothrow) lb_batch();
    if (!b) return bfail(nullptr, LB_ERR_CUDA, "lb_batch_create: out of host memory");
    b->nbox = nbox;
    b->prec = precision;
    b->stream = (cudaStream_t)cuda_stream;
    auto bail = [&](int code) {
        lb_batch_free(b);
        return code;
    };
    cudaError_t e = cudaMalloc((void**)&b->mem, total);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        g_init_err = std::string("lb_batch_create: ") + cudaGetErrorString(e);
        return bail(LB_ERR_CUDA);
    }
    size_t node_off = 0;
    for (int i = 0; i < nbox; ++i) {
        const int nx = dims[3 * i], ny = dims[3 * i + 1], nz = dims[3 * i + 2];
        lb_ctx* c = nullptr;
        const int rc = init_common(&c, nx, ny, nz, precision, rho_r + node_off, rho_b + node_off, cuda_stream,
                                   b->mem + off[i], make_plan(make_layout(nx, ny, nz, precision), precision).total);
        if (rc != LB_OK) return bail(rc);
        b->box.push_back(c);
        if (lb_set_params(c, &params[i]) != LB_OK) {
            g_init_err = "lb_batch_create: box " + std::to_string(i) + ": " + c->err;
            return bail(LB_ERR_ARG);
        }
        node_off += (size_t)nx * ny * nz;
    }
    const int rc = batch_build(b);
    if (rc != LB_OK) {
        g_init_err = b->err;
        return bail(rc);
    }
    *out = b;
    return LB_OK;
}

int lb_batch_set_params(lb_batch* b, int i, const lb_params* params)
{
    if (!b || i < 0 || i >= b->nbox) return bfail(b, LB_ERR_ARG, "lb_batch_set_params: bad argument");
    const int rc = lb_set_params(b->box[i], params);
    if (rc != LB_OK) return bfail(b, rc, b->box[i]->err);
    return batch_build(b);
}

int lb_batch_set_schedule(lb_batch* b, int tile_y, int planes_per_item, int ctas_per_sm)
{
    if (!b || (tile_y != 4 && tile_y != 8 && tile_y != 16) || planes_per_item < 1 || ctas_per_sm < 0)
        return bfail(b, LB_ERR_ARG, "lb_batch_set_schedule: tile_y 4/8/16, planes_per_item >= 1, ctas_per_sm >= 0");
    b->tile_y = tile_y;
    b->seg_planes = planes_per_item;
    b->ctas_per_sm = ctas_per_sm;
    return batch_build(b);
}

int lb_batch_set_step_variant(lb_batch* b, int variant)
{
    if (!b || variant < LB_STEP_AUTO || variant > LB_STEP_TMA)
        return bfail(b, LB_ERR_ARG, "lb_batch_set_step_variant: unknown variant");
    b->variant = variant;
    return batch_build(b);
}

int lb_batch_step(lb_batch* b, int nsteps)
{
    if (!b || nsteps < 0) return bfail(b, LB_ERR_ARG, "lb_batch_step: bad argument");
    for (lb_ctx* c : b->box)
        if (c->cur != b->cur) return bfail(b, LB_ERR_STATE, "lb_batch_step: a box was stepped on its own");
    const int G = lb_ctx::kGraphSteps;
    int n = nsteps;
    if (n >= G) {
        const int par = b->cur;
        if (!b->graph[par]) {
            cudaGraph_t g = nullptr;
            LB_BCUDA(b, cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaSuccess;
            for (int i = 0; i < G && e == cudaSuccess; ++i) e = batch_launch(b, (par + i) & 1, b->cap);
            cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
            if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("lb_batch_step: capture: ") + cudaGetErrorString(e));
            if (e2 != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("lb_batch_step: end capture: ") + cudaGetErrorString(e2));
            e = cudaGraphInstantiate(&b->graph[par], g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return bfail(b, LB_ERR_CUDA, std::string("lb_batch_step: instantiate: ") + cudaGetErrorString(e));
        }
        while (n >= G) {
            LB_BCUDA(b, cudaGraphLaunch(b->graph[par], b->stream));
            n -= G;
        }
    }
    for (int i = 0; i < n; ++i) {
        LB_BCUDA(b, batch_launch(b, b->cur, b->stream));
        b->cur ^= 1;
    }
    b->steps += nsteps;
    for (lb_ctx* c : b->box) {
        c->cur = b->cur;
        c->steps += nsteps;
    }
    return LB_OK;
}

int lb_batch_box(lb_batch* b, int i, lb_ctx** out)
{
    if (!b || !out || i < 0 || i >= b->nbox) return bfail(b, LB_ERR_ARG, "lb_batch_box: bad argument");
    *out = b->box[i];
    return LB_OK;
}

int lb_batch_conservation(lb_batch* b, double* cons)
{
    if (!b || !cons) return bfail(b, LB_ERR_ARG, "lb_batch_conservation: NULL argument");
    for (int i = 0; i < b->nbox; ++i) {
        const int rc = lb_conservation(b->box[i], cons + 8 * (size_t)i);
        if (rc != LB_OK) return bfail(b, rc, "box " + std::to_string(i) + ": " + b->box[i]->err);
    }
    return LB_OK;
}

int lb_batch_contact_angles(lb_batch* b, double offset, lb_droplet* out)
{
    if (!b || !out) return bfail(b, LB_ERR_ARG, "lb_batch_contact_angles: NULL argument");
    for (int i = 0; i < b->nbox; ++i) {
        const int rc = lb_contact_angle(b->box[i], offset, &out[i]);
        if (rc != LB_OK) return bfail(b, rc, "box " + std::to_string(i) + ": " + b->box[i]->err);
    }
    return LB_OK;
}

const char* lb_batch_last_error(const lb_batch* b)
{
    if (!b) return g_init_err.c_str();
    return b->err.c_str();
}

void lb_batch_free(lb_batch* b)
{
    if (!b) return;
    if (b->stream || b->mem) cudaStreamSynchronize(b->stream);
    batch_drop_graphs(b);
    for (lb_ctx* c : b->box) lb_free(c);
    if (b->dargs) cudaFree(b->dargs);
    if (b->ditems) cudaFree(b->ditems);
    if (b->dmaps) cudaFree(b->dmaps);
    if (b->mem) cudaFree(b->mem);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
}

}  // extern "C"

// ====================================================================== adjoint

namespace {
// device allocations of one lb_step_backward call, released on every path
struct AdjScratch {
    std::vector<void*> ptrs;
    ~AdjScratch()
    {
        for (void* p : ptrs) cudaFree(p);
    }
    cudaError_t alloc(void** p, size_t bytes)
    {
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) ptrs.push_back(*p);
        return e;
    }
};
}  // namespace

template <class S>
static cudaError_t adj_step_into(lb_ctx* c, const void* src, void* dst, cudaStream_t st)
{
    StepArgs<S> A = step_args<S>(c, 0);
    A.src = (const S*)src;
    A.dst = (S*)dst;
    return launch_step<S>(A, c->tile_y, c->general, tau_one(c), st);
}

template <class S>
static cudaError_t adj_forward_of(lb_ctx* c, const void* f, const AdjFields& A, cudaStream_t st)
{
    return launch_adj_forward<S>(c->L, c->kp, (const S*)f, A, st);
}

extern "C" int lb_step_backward(lb_ctx* c, int nsteps, int ckpt_every, int observable, double* dJ_deta, double* J)
{
    if (!c || nsteps < 0 || ckpt_every < 1 || observable < 0 || observable > 2 || !dJ_deta)
        return fail(c, LB_ERR_ARG, "lb_step_backward: bad argument");
    if (c->general) return fail(c, LB_ERR_UNSUPPORTED, "lb_step_backward: planar walls only");
    cudaStream_t st = c->stream;
    const long long N = (long long)c->nx * c->ny * c->nz;
    const size_t sb = payload_bytes(c);
    const int nseg = (nsteps + ckpt_every - 1) / ckpt_every;
    const int slen = nsteps < ckpt_every ? (nsteps > 0 ? nsteps : 1) : ckpt_every;
    AdjScratch M;
    char* ck = nullptr;
    char* store = nullptr;
    float* lam = nullptr;
    float* aux = nullptr;
    double* dsc = nullptr;
    if (nseg > 0) LB_CUDA(c, M.alloc((void**)&ck, sb * (size_t)nseg));
    LB_CUDA(c, M.alloc((void**)&store, sb * (size_t)(slen + 1)));
    LB_CUDA(c, M.alloc((void**)&lam, sizeof(float) * 2 * 2 * Q * (size_t)N));
    LB_CUDA(c, M.alloc((void**)&aux, sizeof(float) * 26 * (size_t)N));
    LB_CUDA(c, M.alloc((void**)&dsc, sizeof(double) * (2 * kAdjBlocks + 8)));
    double* part = dsc;
    double* acc = dsc + 2 * kAdjBlocks;
    double* sums = acc + 2;
    AdjFields A;
    {
        float* q = aux;
        for (int a = 0; a < 2; ++a) A.rho[a] = q, q += N;
        for (int a = 0; a < 2; ++a) A.psi[a] = q, q += N;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 3; ++d) A.j[a][d] = q, q += N;
        for (int a = 0; a < 2; ++a) A.rhob[a] = q, q += N;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 3; ++d) A.jb[a][d] = q, q += N;
        for (int a = 0; a < 2; ++a)
            for (int d = 0; d < 3; ++d) A.V[a][d] = q, q += N;
        for (int a = 0; a < 2; ++a) A.psib[a] = q, q += N;
    }
    AdjArgs G;
    G.nx = c->nx;
    G.ny = c->ny;
    G.nz = c->nz;
    G.gk = c->kp.gk;
    for (int k = 0; k < Q; ++k) G.G[k] = k == 0 ? 0.f : (is_axis(k) ? c->kp.Gax : c->kp.Gdi);
    for (int a = 0; a < 2; ++a) {
        G.tau[a] = c->kp.tau[a];
        G.omega[a] = c->kp.itau[a];
        G.eta[a] = c->kp.eta[a];
    }
    auto fwd_on = [&](const void* f, cudaStream_t s2) -> cudaError_t {
        switch (c->prec) {
        case LB_F32: return adj_forward_of<float>(c, f, A, s2);
        case LB_F16: return adj_forward_of<__half>(c, f, A, s2);
        default: return adj_forward_of<__nv_bfloat16>(c, f, A, s2);
        }
    };
    auto fwd = [&](const void* f) { return fwd_on(f, st); };
    auto step_into = [&](const void* src, void* dst, cudaStream_t s2) -> cudaError_t {
        switch (c->prec) {
        case LB_F32: return adj_step_into<float>(c, src, dst, s2);
        case LB_F16: return adj_step_into<__half>(c, src, dst, s2);
        default: return adj_step_into<__nv_bfloat16>(c, src, dst, s2);
        }
    };
    // One segment's recompute and reverse sweep, as launched on stream s2. The
    // launches depend only on the segment length and on which lambda buffer
    // holds lambda(t+1) at its end, so each such pair is captured once into a
    // CUDA graph and replayed (about 5 launches per step otherwise).
    auto segment = [&](int len, float* ln, float* lc, cudaStream_t s2) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < len && e == cudaSuccess; ++i) e = step_into(store + sb * (size_t)i, store + sb * (size_t)(i + 1), s2);
        for (int i = len - 1; i >= 0 && e == cudaSuccess; --i) {
            e = fwd_on(store + sb * (size_t)i, s2);
            if (e == cudaSuccess) e = launch_adj_backstep(G, A, ln, lc, part, acc, s2);
            std::swap(ln, lc);
        }
        return e;
    };
    struct SegGraphs {
        std::vector<std::pair<long long, cudaGraphExec_t>> g;
        ~SegGraphs()
        {
            for (auto& p : g) cudaGraphExecDestroy(p.second);
        }
    } graphs;
    auto run_segment = [&](int len, float* ln, float* lc) -> cudaError_t {
        const long long key = 2LL * len + (ln == lam ? 0 : 1);
        for (auto& p : graphs.g)
            if (p.first == key) return cudaGraphLaunch(p.second, st);
        cudaGraph_t gr = nullptr;
        cudaError_t e = cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        const cudaError_t e1 = segment(len, ln, lc, c->cap);
        e = cudaStreamEndCapture(c->cap, &gr);
        if (e1 != cudaSuccess) e = e1;
        cudaGraphExec_t ex = nullptr;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, gr, 0);
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess) return e;
        graphs.g.emplace_back(key, ex);
        return cudaGraphLaunch(ex, st);
    };

    // forward: a checkpoint at the start of every segment (with the step count,
    // which keys the 16-bit rounding dither, so the recompute replays it)
    std::vector<long long> ck_steps(nseg > 0 ? nseg : 1);
    for (int s = 0; s < nseg; ++s) {
        ck_steps[s] = c->steps;
        LB_CUDA(c, cudaMemcpyAsync(ck + sb * (size_t)s, c->f[c->cur], sb, cudaMemcpyDeviceToDevice, st));
        const int len = nsteps - s * ckpt_every < ckpt_every ? nsteps - s * ckpt_every : ckpt_every;
        const int rc = lb_step(c, len);
        if (rc != LB_OK) return rc;
    }
    // observable of the final state and lambda(T) = dJ/dn(T)
    const double eps = 0.05;
    float* lam_next = lam;
    float* lam_cur = lam + 2 * Q * (size_t)N;
    LB_CUDA(c, fwd(c->f[c->cur]));
    LB_CUDA(c, launch_observable(c->nx, c->ny, c->nz, observable, eps, A.rho[0], A.rho[1], part, sums, lam_next, st));
    LB_CUDA(c, cudaMemsetAsync(acc, 0, 2 * sizeof(double), st));
    // backward, segment by segment: recompute the segment's states, then sweep them in reverse
    for (int s = nseg - 1; s >= 0; --s) {
        const int t0 = s * ckpt_every;
        const int len = nsteps - t0 < ckpt_every ? nsteps - t0 : ckpt_every;
        LB_CUDA(c, cudaMemcpyAsync(store, ck + sb * (size_t)s, sb, cudaMemcpyDeviceToDevice, st));
        LB_CUDA(c, launch_clock_set(c->clock, (uint32_t)ck_steps[s], st));
        LB_CUDA(c, run_segment(len, lam_next, lam_cur));
        if (len & 1) std::swap(lam_next, lam_cur);
    }
    LB_CUDA(c, launch_clock_set(c->clock, (uint32_t)c->steps, st));
    double h[3] = {0, 0, 0};
    LB_CUDA(c, cudaMemcpyAsync(h, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    LB_CUDA(c, cudaMemcpyAsync(h + 2, sums + 2, sizeof(double), cudaMemcpyDeviceToHost, st));
    LB_CUDA(c, cudaStreamSynchronize(st));
    dJ_deta[0] = h[0];
    dJ_deta[1] = h[1];
    if (J) *J = h[2];
    return check_device_status(c);
}

extern "C" int lb_observable(lb_ctx* c, int observable, double* J)
{
    if (!c || !J || observable < 0 || observable > 2) return fail(c, LB_ERR_ARG, "lb_observable: bad argument");
    if (c->general) return fail(c, LB_ERR_UNSUPPORTED, "lb_observable: planar walls only");
    const long long N = (long long)c->nx * c->ny * c->nz;
    AdjScratch M;
    float* aux = nullptr;
    double* dsc = nullptr;
    LB_CUDA(c, M.alloc((void**)&aux, sizeof(float) * 10 * (size_t)N));
    LB_CUDA(c, M.alloc((void**)&dsc, sizeof(double) * (2 * kAdjBlocks + 8)));
    AdjFields A{};
    float* q = aux;
    for (int a = 0; a < 2; ++a) A.rho[a] = q, q += N;
    for (int a = 0; a < 2; ++a) A.psi[a] = q, q += N;
    for (int a = 0; a < 2; ++a)
        for (int d = 0; d < 3; ++d) A.j[a][d] = q, q += N;
    cudaError_t e;
    switch (c->prec) {
    case LB_F32: e = adj_forward_of<float>(c, c->f[c->cur], A, c->stream); break;
    case LB_F16: e = adj_forward_of<__half>(c, c->f[c->cur], A, c->stream); break;
    default: e = adj_forward_of<__nv_bfloat16>(c, c->f[c->cur], A, c->stream); break;
    }
    LB_CUDA(c, e);
    LB_CUDA(c, launch_observable(c->nx, c->ny, c->nz, observable, 0.05, A.rho[0], A.rho[1], dsc,
                                 dsc + 2 * kAdjBlocks, nullptr, c->stream));
    LB_CUDA(c, cudaMemcpyAsync(J, dsc + 2 * kAdjBlocks + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    return LB_OK;
}

// ---------------------------------------------------------------- pressure tensor and surface tension
template <class S>
static cudaError_t pressure_field_of(lb_ctx* c, double* out)
{
    return launch_pressure_field<S>(field_args(c), (const S*)c->f[c->cur], c->W, out, c->stream);
}
template <class S>
static cudaError_t pressure_planes_of(lb_ctx* c, double* out)
{
    return launch_pressure_planes<S>(field_args(c), (const S*)c->f[c->cur], c->W, out, c->stream);
}

extern "C" int lb_pressure_tensor(lb_ctx* c, double* P)
{
    if (!c || !P) return fail(c, LB_ERR_ARG, "lb_pressure_tensor: NULL argument");
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    AdjScratch M;
    double* d = nullptr;
    LB_CUDA(c, M.alloc((void**)&d, 6 * N * sizeof(double)));
    LB_CUDA(c, dispatch_fields(c, true));
    switch (c->prec) {
    case LB_F32: LB_CUDA(c, pressure_field_of<float>(c, d)); break;
    case LB_F16: LB_CUDA(c, pressure_field_of<__half>(c, d)); break;
    default: LB_CUDA(c, pressure_field_of<__nv_bfloat16>(c, d)); break;
    }
    LB_CUDA(c, cudaMemcpyAsync(P, d, 6 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    return LB_OK;
}

extern "C" int lb_pressure_profile(lb_ctx* c, double* prof, double* gamma_sum)
{
    if (!c || !prof) return fail(c, LB_ERR_ARG, "lb_pressure_profile: NULL argument");
    const int nz = c->nz;
    AdjScratch M;
    double* d = nullptr;
    LB_CUDA(c, M.alloc((void**)&d, (size_t)nz * 8 * sizeof(double)));
    LB_CUDA(c, dispatch_fields(c, true));
    switch (c->prec) {
    case LB_F32: LB_CUDA(c, pressure_planes_of<float>(c, d)); break;
    case LB_F16: LB_CUDA(c, pressure_planes_of<__half>(c, d)); break;
    default: LB_CUDA(c, pressure_planes_of<__nv_bfloat16>(c, d)); break;
    }
    LB_CUDA(c, cudaMemcpyAsync(prof, d, (size_t)nz * 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    // sums -> plane means; Eq. gammaMechDef with P_N = P_zz, P_T = (P_xx + P_yy)/2, dz = 1
    double g = 0.0;
    for (int z = 0; z < nz; ++z) {
        double* p = prof + (size_t)z * 8;
        const double n = p[7];
        if (n > 0) {
            for (int v = 0; v < 7; ++v) p[v] /= n;
            g += p[2] - 0.5 * (p[0] + p[1]);
        }
    }
    if (gamma_sum) *gamma_sum = g;
    return LB_OK;
}

extern "C" int lb_pressure_radial(lb_ctx* c, const double* centre, double dr, int nbins, double zmin, double r_max,
                                  double* bins, double* gamma, double* R_s)
{
    if (!c || !centre || !bins || !(dr > 0) || nbins < 1 || nbins > kRadialBinsMax || !std::isfinite(zmin) ||
        !std::isfinite(r_max) || !std::isfinite(centre[0]) || !std::isfinite(centre[1]) || !std::isfinite(centre[2]))
        return fail(c, LB_ERR_ARG, "lb_pressure_radial: bad argument (dr > 0, 1 <= nbins <= 1024, finite centre)");
    AdjScratch M;
    unsigned long long* d = nullptr;
    LB_CUDA(c, M.alloc((void**)&d, (size_t)nbins * 4 * sizeof(unsigned long long)));
    LB_CUDA(c, dispatch_fields(c, true));
    LB_CUDA(c, launch_pressure_radial(field_args(c), c->f[c->cur], c->prec, c->W, centre, dr, nbins, zmin, d,
                                      c->stream));
    std::vector<unsigned long long> h((size_t)nbins * 4);
    LB_CUDA(c, cudaMemcpyAsync(h.data(), d, h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    LB_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int b = 0; b < nbins; ++b) {
        const double n = (double)h[(size_t)b * 4 + 3];
        for (int v = 0; v < 3; ++v) {
            const double sum = (double)(long long)h[(size_t)b * 4 + v] / kRadialFix;
            bins[(size_t)b * 4 + v] = n > 0 ? sum / n : 0.0;
        }
        bins[(size_t)b * 4 + 3] = n;
    }
    // Eq. mechRadGamma: R_s where the bin-mean phi first changes sign going
    // outward (linear between bin centres), then sum (r_b/R_s)^2 (P_N - P_T) dr
    double rs = std::nan("");
    int prev = -1;
    for (int b = 0; b < nbins; ++b) {
        if (bins[(size_t)b * 4 + 3] == 0) continue;
        if (prev >= 0 && (bins[(size_t)prev * 4 + 2] > 0) != (bins[(size_t)b * 4 + 2] > 0)) {
            const double r0 = (prev + 0.5) * dr, r1 = (b + 0.5) * dr;
            const double p0 = bins[(size_t)prev * 4 + 2], p1 = bins[(size_t)b * 4 + 2];
            rs = r0 + (r1 - r0) * p0 / (p0 - p1);
            break;
        }
        prev = b;
    }
    double g = 0.0;
    if (rs == rs)
        for (int b = 0; b < nbins; ++b) {
            const double rb = (b + 0.5) * dr;
            if (bins[(size_t)b * 4 + 3] > 0 && rb <= r_max)
                g += (rb / rs) * (rb / rs) * (bins[(size_t)b * 4 + 0] - bins[(size_t)b * 4 + 1]) * dr;
        }
    if (gamma) *gamma = g;
    if (R_s) *R_s = rs;
    return LB_OK;
}

// ---------------------------------------------------------------- closed forms of the contact angle
static double clamp_acos_deg(double c)
{
    c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
    return std::acos(c) * 180.0 / 3.14159265358979323846;
}

extern "C" int lb_young_theta(double gamma_sg, double gamma_sl, double gamma_lg, double* theta_deg)
{
    if (!theta_deg || !std::isfinite(gamma_sg) || !std::isfinite(gamma_sl) || !std::isfinite(gamma_lg) ||
        !(gamma_lg > 0)) {
        lbsc_set_global_error("lb_young_theta: finite tensions and gamma_lg > 0 required");
        return LB_ERR_ARG;
    }
    *theta_deg = clamp_acos_deg((gamma_sg - gamma_sl) / gamma_lg);
    return LB_OK;
}

extern "C" int lb_huang_theta(double eta_wall_r, double eta_wall_b, double rho_in, double rho_out, double* theta_deg)
{
    if (!theta_deg || !std::isfinite(eta_wall_r) || !std::isfinite(eta_wall_b) || !std::isfinite(rho_in) ||
        !std::isfinite(rho_out) || !(rho_in > rho_out)) {
        lbsc_set_global_error("lb_huang_theta: finite arguments and rho_in > rho_out required");
        return LB_ERR_ARG;
    }
    // G_ads of the r droplet's own component is g eta_wall_b (the wall as felt by r), that of the
    // surrounding b component g eta_wall_r; g cancels against the denominator g (rho_in - rho_out)/2
    *theta_deg = clamp_acos_deg((eta_wall_r - eta_wall_b) / (0.5 * (rho_in - rho_out)));
    return LB_OK;
}

// ---------------------------------------------------------------- 16-bit rounding self-test
extern "C" int lb_selftest_round(int precision, const float* v, const unsigned* m, int n, unsigned* out)
{
    if ((precision != LB_F16 && precision != LB_BF16) || !v || !m || !out || n < 1 || n > (1 << 24)) {
        lbsc_set_global_error("lb_selftest_round: LB_F16 or LB_BF16, host arrays and 1 <= n <= 2^24 required");
        return LB_ERR_ARG;
    }
    float* dv = nullptr;
    uint32_t* du = nullptr;
    cudaError_t e = cudaMalloc(&dv, (size_t)2 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&du, (size_t)4 * n * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMemcpy(dv, v, (size_t)2 * n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(du, m, (size_t)n * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = lbsc::launch_round_probe(precision == LB_F16 ? 1 : 2, dv, du, n, du + n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, du + n, (size_t)3 * n * sizeof(uint32_t), cudaMemcpyDeviceToHost);
    for (void* p : {(void*)dv, (void*)du})
        if (p) {
            const cudaError_t f = cudaFree(p);
            if (e == cudaSuccess) e = f;
        }
    if (e != cudaSuccess) {
        lbsc_set_global_error(std::string("lb_selftest_round: ") + cudaGetErrorString(e));
        return LB_ERR_CUDA;
    }
    return LB_OK;
}

// ---------------------------------------------------------------- psi self-test
extern "C" int lb_selftest_psi(const float* rho, int n, float* out)
{
    if (!rho || !out || n < 1 || n > (1 << 24)) {
        lbsc_set_global_error("lb_selftest_psi: host arrays and 1 <= n <= 2^24 required");
        return LB_ERR_ARG;
    }
    float* d = nullptr;
    cudaError_t e = cudaMalloc(&d, (size_t)5 * n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(d, rho, (size_t)n * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = lbsc::launch_psi_probe(d, n, d + n, nullptr);
    if (e == cudaSuccess) e = cudaMemcpy(out, d + n, (size_t)4 * n * sizeof(float), cudaMemcpyDeviceToHost);
    if (d) {
        const cudaError_t f = cudaFree(d);
        if (e == cudaSuccess) e = f;
    }
    if (e != cudaSuccess) {
        lbsc_set_global_error(std::string("lb_selftest_psi: ") + cudaGetErrorString(e));
        return LB_ERR_CUDA;
    }
    return LB_OK;
}
