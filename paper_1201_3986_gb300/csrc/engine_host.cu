// Host side of the generic engine: workspace layout, item split, launches.
#include <algorithm>

#include "engine.cuh"

qdvm_status moments_batched_launch(const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                                   const void* Q, int prec, double* m, cudaStream_t st);

namespace eng {
namespace {

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

int occupancy(int mode, int prec, int d, int zc, bool stage, size_t smem) {
    if (mode == FWD) return occupancy_fwd(prec, d, zc, stage, smem);
    if (mode == JVP) return occupancy_jvp(prec, d, zc, stage, smem);
    return occupancy_vjp(prec, d, zc, stage, smem);
}

__global__ void k_single_init(int* counter, int* order, int* cell_plan, int64_t* cell_offset) {
    *counter = 0;
    *order = 0;
    *cell_plan = 0;
    *cell_offset = 0;
}

template <typename T, bool KAHAN>
void reduce(const Layout& g, const BatchDev& b, int n_cells, const int* cp, const int64_t* co, char* base, void* out,
            cudaStream_t st) {
    dim3 grid(8, std::max(1, std::min(n_cells, 65535)));
    k_reduce_chunks<T, KAHAN><<<grid, 256, 0, st>>>(b, n_cells, g.C, cp, co,
                                                     reinterpret_cast<const T*>(base + g.off_part), g.part_stride,
                                                     static_cast<T*>(out));
}

}  // namespace

Layout make_layout(int mode, const BatchDev& b, int n_cells, int prec, bool single, int chunks) {
    Layout g{};
    g.mode = mode;
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    const bool kahan = prec == QDVM_F32_KAHAN;
    int maxLines = 0, zc = 8, d = 2;
    size_t padn = 0, nn = 0;
    for (int i = 0; i < b.n_plans; ++i) {
        const int N = b.p[i].N, H = b.p[i].Ntilde;
        d = b.p[i].d;
        const size_t S = d == 3 ? (size_t)N * N : (size_t)N;
        maxLines = std::max(maxLines, b.p[i].n_lines);
        padn = std::max(padn, (size_t)(N + 2 * H) * S);
        nn = std::max(nn, S * N);
        if (N % 8) zc = 1;
    }
    g.d = d;
    g.zc = zc;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    g.stage = padn * es + 4096 <= (size_t)optin;
    g.smem = g.stage ? padn * es : 0;
    const int per = occupancy(mode, prec, d, zc, g.stage, g.smem);
    const int slots = per * qdvm_num_sms();
    const int nc = std::max(n_cells, 1);
    if (single)
        g.C = std::max(1, std::min(maxLines, slots));
    else
        g.C = std::max(1, std::min(maxLines, (4 * slots + nc - 1) / nc));
    if (!single && nc >= 2 * slots) g.C = 1;
    if (chunks > 0) g.C = std::max(1, std::min(maxLines, chunks));
    const long items = (long)nc * g.C;
    g.grid = (int)std::max(1L, std::min(items, (long)slots));
    g.scr_stride = a256(((size_t)n_fields(mode, g.stage) * padn + (kahan ? nn : 0)) * es);
    g.part_stride = g.C > 1 ? nn : 0;
    g.off_scr = 256 + a256((size_t)nc * sizeof(int)) + 256;  // counter, order, single-cell tables
    g.off_part = g.off_scr + (size_t)g.grid * g.scr_stride;
    g.total = g.off_part + (g.C > 1 ? a256((size_t)nc * g.C * nn * es) : 0);
    return g;
}

}  // namespace eng

size_t engine_workspace(int mode, const BatchDev& b, int n_cells, int prec, bool single, int chunks) {
    return eng::make_layout(mode, b, single ? 1 : n_cells, prec, single, chunks).total;
}

qdvm_status engine_run(int mode, const BatchDev& b, int n_cells, const int* cell_plan, const int64_t* cell_offset,
                       const void* f, const void* aux, void* out, double* moments, int prec, void* ws,
                       size_t ws_bytes, bool single, int chunks, cudaStream_t st) {
    using namespace eng;
    const int nc = single ? 1 : n_cells;
    const Layout g = make_layout(mode, b, nc, prec, single, chunks);
    if (!ws || ws_bytes < g.total) return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for the line engine");
    char* base = static_cast<char*>(ws);
    int* counter = reinterpret_cast<int*>(base);
    int* order = reinterpret_cast<int*>(base + 256);
    if (single) {
        char* tab = base + 256 + 256;
        int* cp = reinterpret_cast<int*>(tab);
        int64_t* co = reinterpret_cast<int64_t*>(tab + 128);
        k_single_init<<<1, 1, 0, st>>>(counter, order, cp, co);
        QDVM_LAUNCH_CHECK("engine single init");
        cell_plan = cp;
        cell_offset = co;
    } else {
        qdvm_status s = schedule_launch(b, nc, cell_plan, order, counter, st);
        if (s != QDVM_OK) return s;
    }
    qdvm_status s;
    if (mode == FWD) s = launch_fwd(g, b, nc, cell_plan, cell_offset, order, counter, f, aux, out, base, prec, st);
    else if (mode == JVP) s = launch_jvp(g, b, nc, cell_plan, cell_offset, order, counter, f, aux, out, base, prec, st);
    else s = launch_vjp(g, b, nc, cell_plan, cell_offset, order, counter, f, aux, out, base, prec, st);
    if (s != QDVM_OK) return s;
    if (g.C > 1) {
        if (prec == QDVM_F64) reduce<double, false>(g, b, nc, cell_plan, cell_offset, base, out, st);
        else if (prec == QDVM_F32_KAHAN) reduce<float, true>(g, b, nc, cell_plan, cell_offset, base, out, st);
        else reduce<float, false>(g, b, nc, cell_plan, cell_offset, base, out, st);
        QDVM_LAUNCH_CHECK("engine reduce launch");
    }
    if (moments) return moments_batched_launch(b, nc, cell_plan, cell_offset, out, prec, moments, st);
    return QDVM_OK;
}
