// Host side of the fused 2D evaluator: shared-memory sizing, support test,
// workspace, and the dispatch to the per-precision translation units.  The
// kernels themselves are in fused2d.cuh.
#include "fused2d.cuh"

size_t fused2d_smem_bytes(int N, int H, int prec, int fft) {
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    size_t b = (buf_f_elems(N, H) + buf_p_elems(N, H)) * es;
    if (fft) {
        // the FFT body's layouts for the compile-time cell sizes (GeoF):
        // without SCAN the cell with an H halo (with the STAIR point map of
        // FP32 cells, XR more columns and an odd stride, largest over the
        // CTA sizes) followed by the FFT buffers; with SCAN the cell with a
        // 2H halo and the two window fields, the FFT buffers aliasing them
        int xr = 0;
        if (prec != QDVM_F64 && N == 64) xr = std::max(body_xr<float, 64, 256>(), body_xr<float, 64, 512>());
        if (prec != QDVM_F64 && N == 32)
            xr = std::max({body_xr<float, 32, 128>(), body_xr<float, 32, 256>(), body_xr<float, 32, 512>()});
        const size_t W = N + 2 * H, LD = N + 1;
        size_t RS = W + (((N % 32) - (W % 32) + 32) % 32);
        if (xr) RS = std::max(RS, (W + xr) | 1);
        const size_t fftb = 2 * (size_t)N * LD * 2 * es;
        const size_t direct = (W * RS * es + 15) / 16 * 16 + fftb;
        const size_t scan = std::max(fftb, (buf_f_elems(N, H) * es + 15) / 16 * 16 + 2 * (size_t)N * N * es);
        b = std::max(b, std::max(direct, scan));
    }
    return b;
}

int fused2d_supported(int N, int H, int prec) {
    if (N * N > 16 * 256) return 0;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return fused2d_smem_bytes(N, H, prec, 1) + 2048 <= (size_t)optin;
}

size_t fused2d_single_workspace(const qdvm_plan_s* p, int prec) {
    int S, ppc;
    split_pairs(p->n_pairs, qdvm_num_sms(), &S, &ppc);
    if (S <= 1) return 0;
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    return (size_t)S * p->N * p->N * es;
}

qdvm_status fused2d_eval_single(const qdvm_plan_s* p, const void* f, void* Q, int prec, void* ws, size_t ws_bytes,
                                cudaStream_t st) {
    int S, ppc;
    split_pairs(p->n_pairs, qdvm_num_sms(), &S, &ppc);
    const size_t need = fused2d_single_workspace(p, prec);
    if (need > 0 && (ws == nullptr || ws_bytes < need))
        return qdvm_fail(QDVM_ERR_INVALID_ARG, "workspace too small for qdvm_eval");
    const size_t smem = fused2d_smem_bytes(p->N, p->Ntilde, prec, p->tune.loss_fft);
    switch (prec) {
        case QDVM_F64: return fused2d_single_f64(p, f, Q, ws, S, ppc, smem, st);
        case QDVM_F32: return fused2d_single_f32(p, f, Q, ws, S, ppc, smem, st);
        default: return fused2d_single_f32k(p, f, Q, ws, S, ppc, smem, st);
    }
}

// Shared memory of the batched evaluator's CTA for one plan: the layout of
// the FFT body (body_smem) for the cell sizes it is compiled for, when the
// plan runs it (loss_fft set, the loss kernel's transform present); the
// buffers of the line-engine body otherwise.
static size_t batched_plan_smem(const PlanDev& p, int prec, int threads) {
    const int N = p.N, H = p.Ntilde, fft = p.tfft, sj = p.tsj;
    if (fft && p.khat) {
#define QDVM_BODY_SMEM(NN, HH)                                                                       \
    if (N == NN && H == HH) {                                                                        \
        if (prec == QDVM_F64)                                                                        \
            return threads == 512 ? body_smem<double, NN, HH, 512>(fft, sj)                          \
                                  : body_smem<double, NN, HH, 256>(fft, sj);                         \
        return threads == 512 ? body_smem<float, NN, HH, 512>(fft, sj) : body_smem<float, NN, HH, 256>(fft, sj); \
    }
        QDVM_BODY_SMEM(64, 14)
        QDVM_BODY_SMEM(48, 10)
        QDVM_BODY_SMEM(32, 7)
        QDVM_BODY_SMEM(16, 3)
#undef QDVM_BODY_SMEM
    }
    const size_t es = prec == QDVM_F64 ? sizeof(double) : sizeof(float);
    return (buf_f_elems(N, H) + buf_p_elems(N, H)) * es;
}

qdvm_status fused2d_eval_batched(const BatchDev& b, const qdvm_tuning& tu, int n_cells, const int* cell_plan,
                                 const int64_t* cell_offset, const void* f, void* Q, double* moments, int prec,
                                 void* ws, cudaStream_t st) {
    // workspace: [counter (int, padded to 256 B)] [order: n_cells ints]
    int* counter = static_cast<int*>(ws);
    int* order = reinterpret_cast<int*>(static_cast<char*>(ws) + 256);
    qdvm_status s = schedule_launch(b, n_cells, cell_plan, order, counter, st);
    if (s != QDVM_OK) return s;
    // each cell runs with its plan's own launch parameters (PlanDev); the
    // block size is tu's
    size_t smem = 0;
    for (int i = 0; i < b.n_plans; ++i) {
        smem = std::max(smem, batched_plan_smem(b.p[i], prec, tu.threads));
        // small FP32 cells go several at a time on 256 threads (cell_groups)
        if (prec != QDVM_F64 && tu.threads == 256)
            smem = std::max(smem, group_smem_bytes<float>(cell_groups<float, 256>(
                                      b.p[i].N, b.p[i].Ntilde, b.p[i].khat != nullptr, b.p[i].tfft, b.p[i].tsj)));
    }
    switch (prec) {
        case QDVM_F64:
            return fused2d_batched_f64(b, tu, n_cells, cell_plan, cell_offset, order, counter, f, Q, moments, smem,
                                       st);
        case QDVM_F32:
            return fused2d_batched_f32(b, tu, n_cells, cell_plan, cell_offset, order, counter, f, Q, moments, smem,
                                       st);
        default:
            return fused2d_batched_f32k(b, tu, n_cells, cell_plan, cell_offset, order, counter, f, Q, moments, smem,
                                        st);
    }
}
