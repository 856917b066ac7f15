// static_scratch.cu -- spinsim_simulate_static: one simulation without any
// device or host allocation by the library.
//
// Some callers cannot let a library allocate: real-time control loops where a
// cudaMalloc/cudaFree would synchronise the device and stall an unrelated
// pipeline, frameworks that have already partitioned all device memory with
// their own pooled allocator (a cudaMalloc fails or fragments it), and hosts
// that must not allocate while building their own work.  For them this entry
// point runs the same kernels as spinsim_simulate, with all of its scratch
// (parameter table, sample operators, chain aggregates) in one file-scope
// device array of fixed size.  The caller passes device buffers for the
// outputs and a stream; nothing else is created.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "bounds.cuh"
#include "internal.h"
#include "spinsim.h"

using namespace spinsim;

namespace {

// 16 MiB: a spin-one request of up to ~99,000 output samples (a spin-half
// one of up to ~460,000) fits.  Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t kStaticScratchBytes = size_t(16) << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};   // device address of g_static_scratch, per device


size_t up256(size_t x) { return (x + 255) / 256 * 256; }

bool device_resident(const void* p)
{
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Everything the kernels read from the parameter table, passed by value to a
// set-up kernel that writes it into the static array: no host staging buffer
// and no copy from pageable memory.
struct StaticTable {
    DevSim sim;
    int64_t K;
    int64_t nodes[kMaxLevels];
    int32_t levels;
};

__global__ void static_table_kernel(StaticTable t, DevSim* sims, int64_t* sample_offsets, int64_t* level_off,
                                    unsigned long long* tile_counter)
{
    // the record as 8-byte words, one per thread in turn
    const uint64_t* src = reinterpret_cast<const uint64_t*>(&t.sim);
    uint64_t* dst = reinterpret_cast<uint64_t*>(sims);
    for (int i = threadIdx.x; i < (int)(sizeof(DevSim) / sizeof(uint64_t)); i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) {
        sample_offsets[0] = 0;
        sample_offsets[1] = t.K;
        for (int l = 0; l < t.levels; l++) {
            level_off[2 * l] = 0;
            level_off[2 * l + 1] = t.nodes[l];
        }
        *tile_counter = 0;   // the previous call left its final count here
    }
}
static_assert(sizeof(DevSim) % sizeof(uint64_t) == 0, "DevSim is copied as 8-byte words");

// Restores the caller's current device when the entry point returns.
struct DeviceGuard {
    int prev = -1;
    DeviceGuard()
    {
        if (cudaGetDevice(&prev) != cudaSuccess) {
            cudaGetLastError();
            prev = -1;
        }
    }
    ~DeviceGuard()
    {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

#ifdef SPINSIM_BOUNDS
namespace spinsim {
SPINSIM_BOUNDS_READER(bounds_word_static)
}
#endif

extern "C" int spinsim_simulate_static(const spinsim_config* cfg, const spinsim_request* req, spinsim_result* res,
                                       void* stream_v)
{
    if (!cfg || !req || !res) return SPINSIM_E_ARG;
    if (cfg->method < 0 || cfg->method > 2 || cfg->precision < 0 || cfg->precision > 1 ||
        cfg->trotter_squares < -1 || cfg->trotter_squares > 40 ||
        !(cfg->lanes_per_sample == 0 || cfg->lanes_per_sample == 1 || cfg->lanes_per_sample == 2 ||
          cfg->lanes_per_sample == 4 || cfg->lanes_per_sample == 8) ||
        !(cfg->threads_per_block == 0 || cfg->threads_per_block == 64 || cfg->threads_per_block == 128 ||
          cfg->threads_per_block == 256) ||
        cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 32 || cfg->chain_precision < 0 || cfg->chain_precision > 1)
        return SPINSIM_E_ARG;
    int64_t K = 0, L = 0;
    int st = spinsim_counts(req, &K, &L);
    res->status = st;
    res->flags = 0;
    res->trotter_squares = 0;
    res->n_samples = 0;
    if (st != SPINSIM_OK) return st;
    st = precision_status(*cfg, *req);
    if (st != SPINSIM_OK) return res->status = st;
    res->flags = magnus_flags(*req, L) | precision_flags(cfg->precision, cfg->rotating_frame, *req);
    if (!res->states || res->capacity < K) {
        res->status = !res->states ? SPINSIM_E_ARG : SPINSIM_E_CAPACITY;
        return res->status;
    }
    // outputs must already be device memory (staging would need an allocation)
    const void* outs[3] = {res->states, res->spin, res->ops};
    for (const void* p : outs)
        if (p && (!device_resident(p) || ((uintptr_t)p & 15u) != 0)) {
            res->status = SPINSIM_E_ARG;
            return SPINSIM_E_ARG;
        }
    if (cfg->device < 0 || cfg->device >= kMaxDevices) return res->status = SPINSIM_E_ARG;
    DeviceGuard keep_device;   // the caller's current device is restored on return
    if (cudaSetDevice(cfg->device) != cudaSuccess) return res->status = SPINSIM_E_CUDA;
    // set-up, once per device with that device current: the device address of
    // the static array (its host-side name is not a device address)
    void* base_v = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_addr[cfg->device]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return res->status = SPINSIM_E_CUDA;
            }
            g_scratch_addr[cfg->device] = p;
        }
        base_v = g_scratch_addr[cfg->device];
    }
    char* base = static_cast<char*>(base_v);
    const int spin = req->spin_x2;
    const int opd = op_doubles(spin);
    const ChainGeom cg = chain_geom(K);
    const ChainLayout cl = chain_layout(spin, cg.nodes, cg.top + 1);
    size_t off = 0;
    const size_t sims_off = off; off += up256(sizeof(DevSim));
    const size_t soff_off = off; off += 256;
    const size_t loff_off = off; off += up256(kMaxLevels * 2 * sizeof(int64_t));
    const size_t counter_off = off; off += 256;
    const int variant = request_variant(*cfg, *req, K, L);
    // operator slots: the paired kernels place an odd K's pairs in K + 1 slots
    const int64_t slots = variant_pairs(spin, cfg->precision, variant) ? pair_slots(K) : K;
    const size_t U_off = off; off += up256((size_t)slots * opd * 8);
    const int64_t phase_n = phasor_entries(K, req->field.n_tones);
    const size_t phase_off = off; off += up256((size_t)phase_n * 2 * sizeof(double));
    const size_t chain_off = off; off += cl.bytes;
    if (off > kStaticScratchBytes) return res->status = SPINSIM_E_NOMEM;   // K beyond the static maximum

    const int tau = cfg->trotter_squares;   // -1: chosen per request, as in spinsim_simulate
    DevSim d;
    fill_devsim(*cfg, *req, K, L, d);
    d.states = res->states;
    d.spin = res->spin;
    d.ops = res->ops;
    d.sample_offset = 0;
    d.eb_tab = reinterpret_cast<const double*>(base + phase_off);
    d.eb_off = 0;
    d.chain_run = cg.run;
    d.chain_top = cg.top;
    res->trotter_squares = d.tau;
    // the parameter table (the record, sample offsets {0, K}, per chain level
    // the node offsets {0, nodes}) and a cleared tile counter, written on the
    // stream by one small kernel from its by-value argument
    StaticTable tbl;
    tbl.sim = d;
    tbl.K = K;
    tbl.levels = cg.top + 1;
    for (int l = 0; l < kMaxLevels; l++) tbl.nodes[l] = l <= cg.top ? cg.nodes[l] : 0;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    static_table_kernel<<<1, 32, 0, stream>>>(tbl, reinterpret_cast<DevSim*>(base + sims_off),
                                              reinterpret_cast<int64_t*>(base + soff_off),
                                              reinterpret_cast<int64_t*>(base + loff_off),
                                              reinterpret_cast<unsigned long long*>(base + counter_off));
    if (cudaGetLastError() != cudaSuccess) return res->status = SPINSIM_E_CUDA;
    if (K > 0) {
        int n_sm = 0;
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, cfg->device);
        const int lanes = cfg->lanes_per_sample ? cfg->lanes_per_sample : 1;
        const int block = cfg->threads_per_block ? cfg->threads_per_block : 128;
        int per_sm = 0;
        if (integrate_occupancy(spin, cfg->precision, cfg->method, block, variant, &per_sm) != cudaSuccess) {
            cudaGetLastError();
            return res->status = SPINSIM_E_CUDA;
        }
        if (launch_phase_table(reinterpret_cast<const DevSim*>(base + sims_off), 1, phase_n,
                               reinterpret_cast<double*>(base + phase_off), n_sm, stream) != cudaSuccess)
            return res->status = SPINSIM_E_CUDA;
        IntegrateArgs ia;
        ia.sims = reinterpret_cast<const DevSim*>(base + sims_off);
        ia.sample_offsets = reinterpret_cast<const int64_t*>(base + soff_off);
        ia.n_sims = 1;
        ia.total_samples = slots;
        ia.U = reinterpret_cast<double*>(base + U_off);
        ia.tau = tau;
        ia.tile_counter = reinterpret_cast<unsigned long long*>(base + counter_off);
        if (cfg->blocks_per_sm > 0) per_sm = std::min(per_sm, cfg->blocks_per_sm);
        const int64_t wave_blocks = (int64_t)n_sm * std::max(per_sm, 1);
        integrate_tiles(slots, lanes, block, wave_blocks, seg_log2_of(L), ia,
                        variant_pairs(spin, cfg->precision, variant) ? 2 : 1);
        const int grid =
            (int)std::max<int64_t>(1, std::min<int64_t>((ia.n_tiles + block / 32 - 1) / (block / 32), wave_blocks));
        if (launch_integrate(spin, cfg->precision, cfg->method, block, grid, variant, ia, stream, phase_n > 0) !=
            cudaSuccess)
            return res->status = SPINSIM_E_CUDA;
        ChainArgs ca;
        ca.sims = ia.sims;
        ca.n_sims = 1;
        ca.level_off = reinterpret_cast<const int64_t*>(base + loff_off);
        ca.U = ia.U;
        chain_args_set(ca, cl, base + chain_off);
        ca.max_run = cg.run;
        int chain_k = 0;
        if (launch_chain(spin, ca, n_sm, stream, &chain_k, cfg->chain_precision == 1) != cudaSuccess)
            return res->status = SPINSIM_E_CUDA;
    }
    res->n_samples = K;
    res->status = SPINSIM_OK;
    return SPINSIM_OK;
}
