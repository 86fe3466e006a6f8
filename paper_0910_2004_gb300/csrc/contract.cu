// Contraction of one level (Section 2): the per-phase kernels over the
// device functions of contract.cuh, and their launchers.
#include <algorithm>

#include "contract.cuh"

namespace kp {

// 4 resident blocks per SM (64 registers) measured best for the small rows
__global__ void __launch_bounds__(CONTRACT_BLOCK, 4) k_contract_small(DevState *st, int level, Work w) {
    phase_contract_small(st, level, w);
}

__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_rows32(DevState *st, int level, Work w) {
    phase_contract_rows32(st, level, w);
}

__global__ void __launch_bounds__(CONTRACT_BLOCK) k_contract_overflow(DevState *st, int level, Work w) {
    __shared__ OverflowSmem sm;
    // 2 radix entries per thread and chunk keep the kernel at 48 registers,
    // so the many-warp classes run at full occupancy and the classes overlap
    phase_contract_overflow<true, true, 2, false>(st, level, w, sm);
}

__global__ void k_compact(DevState *st, int level, Work w) { phase_compact(st, level, w); }

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
kp_status launch_relabel(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    const int64_t tiles = scan_tiles(std::max<int64_t>(1, L.n_bound));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 4));
    if (L.matcher == KP_MATCHER_SUITOR) {
        RelabelOp<true> op;
        op.st = L.st;
        op.level = L.level;
        op.w = L.w;
        k_scan_lb<RelabelOp<true>><<<grid, SCAN_BLOCK, 0, s>>>(op, L.w.status, L.epoch_relabel, L.w.spin_limit);
    } else {
        RelabelOp<false> op;
        op.st = L.st;
        op.level = L.level;
        op.w = L.w;
        k_scan_lb<RelabelOp<false>><<<grid, SCAN_BLOCK, 0, s>>>(op, L.w.status, L.epoch_relabel, L.w.spin_limit);
    }
    *launches += 1;
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

kp_status launch_contract(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    const int64_t want = ((int64_t)std::max<int32_t>(1, L.n_bound) + CONTRACT_BLOCK - 1) / CONTRACT_BLOCK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)1 << 30));
    k_contract_small<<<grid, CONTRACT_BLOCK, 0, s>>>(L.st, L.level, L.w);
    // rows of 17..32 entries: one thread each when there are many of them
    // (decided on the device from the class count), else a warp each
    k_contract_rows32<<<num_sms() * 8, CONTRACT_BLOCK, 0, s>>>(L.st, L.level, L.w);
    k_contract_overflow<<<num_sms() * 8, CONTRACT_BLOCK, 0, s>>>(L.st, L.level, L.w);
    *launches += 3;
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

kp_status launch_csr(const LevelLaunch &L, cudaStream_t s, int32_t *launches) {
    const int64_t tiles = scan_tiles(std::max<int64_t>(1, L.n_bound));
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)num_sms() * 4));
    DegScanOp op;
    op.st = L.st;
    op.level = L.level;
    op.w = L.w;
    k_scan_lb<DegScanOp><<<grid, SCAN_BLOCK, 0, s>>>(op, L.w.status, L.epoch_degscan, L.w.spin_limit);
    const int64_t threads = (int64_t)std::max<int32_t>(1, L.n_bound) * 8;
    const int cgrid = (int)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, (int64_t)num_sms() * 16));
    k_compact<<<cgrid, 256, 0, s>>>(L.st, L.level, L.w);
    *launches += 2;
    KP_CUDA(cudaGetLastError());
    return KP_OK;
}

}  // namespace kp
