// spinsim_api.cu -- host engine behind the C ABI of include/spinsim.h.
//
// One batch = validate requests -> plan (sample offsets, chain-tree node
// offsets, parameter table) -> upload the table -> integrate kernel (all U_k) -> chain kernels
// (psi_k, <J>_k, U_k) -> copy back any host-resident outputs.  Requests of
// both spins may share a batch; each spin is one pass of the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <iterator>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "spinsim.h"
#include "internal.h"

using namespace spinsim;

namespace {

bool is_device_pointer(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// -------------------------------------------------------------- scratch
struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

size_t round_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

struct Arena {
    DevBuf buf;   // one allocation carved into the pieces of a batch
};

struct PinnedBuf {
    void* p = nullptr;
    size_t cap = 0;
};

struct Group {
    int spin_x2;
    int variant = kVariantGeneral; // integrate variant of the launch, the same for all its requests
    std::vector<int64_t> idx;      // request indices
    int64_t samples = 0;
    double steps = 0.0;            // CF4 (or sampling) steps of the group
    int min_seg_log2 = kSegLog2;   // smallest canonical segment split among the group's simulations
    int levels = 1;                // chain-tree levels of the tallest simulation
    int max_run = 0;               // the longest chain lane run among the group's simulations
    int64_t nodes[kMaxLevels] = {};  // chain-tree nodes per level, all simulations
    size_t sims_off = 0, soff_off = 0, loff_off = 0, counter_off = 0, U_off = 0, chain_off = 0;
    size_t phase_off = 0;                   // phasor tables of the drives and further tones (FP64 pairs)
    int64_t phase_n = 0;                    // their entries, all simulations of the group
    ChainLayout chain{};
};

struct StagedOut {
    int64_t req;
    double* host_states;
    double* host_spin;
    double* host_ops;
    size_t states_off, spin_off, ops_off;  // offsets into the arena
    size_t states_bytes, spin_bytes, ops_bytes;
};

struct Plan {
    std::vector<Group> groups;
    std::vector<StagedOut> staged;
    std::vector<int64_t> staged_of;   // per request: its entry in `staged`, or -1
    // per request: the addresses the kernels write its outputs to (device
    // memory, or mapped host memory with direct_host_outputs); a staged one is
    // replaced by its piece of the arena when the tables are filled
    std::vector<double*> dev_states, dev_spin, dev_ops;
    size_t total = 0;
    size_t pinned_bytes = 0;
    size_t direct_host_bytes = 0;     // outputs written straight into host memory
};

struct TuneKey {
    int spin, precision, method, tau, variant;
    int64_t size;   // power-of-two bucket of the batch's samples
    bool operator<(const TuneKey& o) const
    {
        return std::tie(spin, precision, method, tau, variant, size) <
               std::tie(o.spin, o.precision, o.method, o.tau, o.variant, o.size);
    }
};
struct TuneVal {
    int lanes, block;
};

// Batches of at most this many CF4 steps are timed on their full size (their
// time depends on how the last wave of tiles fills the GPU, which a prefix
// would not show); larger batches on a prefix of a few waves.  The choice is
// cached per power-of-two size bucket, so a stream of batches of varying size
// (serving) tunes once per bucket.
constexpr double kFullTrialSteps = 4e8;

std::mutex g_tune_mu;
std::map<std::pair<int, TuneKey>, TuneVal> g_tune_cache;   // (device, key) -> choice, shared by handles

}  // namespace

// ------------------------------------------------------------------ handle
struct Ticket {
    spinsim_request req;
    spinsim_result* res;
    int state;    // 0 pending, 1 in flight, 2 done
    int slot;
    size_t bytes;    // scratch of the request alone (staging included)
    size_t staged;   // staging bytes of its host-resident outputs
};

// A serving stream.  Its batch's scratch is a piece [off, off + len) of the
// handle's serving pool, returned to the pool when the batch retires.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<int64_t> tickets;
    size_t off = 0, len = 0;
    PinnedBuf pinned;
};

struct spinsim_s {
    spinsim_config cfg;
    int device = 0;
    int n_sm = 0;
    int tau = 24;
    size_t budget = 0;
    cudaStream_t work = nullptr;    // internal stream (eager runs and graph capture)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_pinned = nullptr;
    // Graph replays run on the caller's stream; ev_done marks the end of the
    // handle's last replay so that the next call, on any stream, starts after it.
    cudaEvent_t ev_done = nullptr;
    bool done_pending = false;
    Arena arena;
    PinnedBuf pinned;
    spinsim_launch_info last{};
    std::map<std::tuple<int, int, int>, int> occ;   // (spin, block, variant) -> resident blocks per SM
    std::vector<char> table_tmp;                     // host copy of the next parameter table
    // graph cache: one batch signature
    std::vector<uint64_t> graph_sig;
    // the last call whose graph was replayed or captured: its requests byte for
    // byte, result buffers and per-request outcome; a call identical to it
    // replays the graph without validating and refilling the tables again
    std::vector<spinsim_request> memo_reqs;
    std::vector<spinsim_result> memo_res;
    cudaGraphExec_t graph_exec = nullptr;
    int graph_kernels = 0;
    int graph_prof_groups = 0;                      // profiled groups whose events the graph records
    spinsim_launch_info graph_info{};
    // profiling: per launch group, events before integrate, after integrate, after chain
    cudaEvent_t prof[kMaxGroups][3] = {};
    int prof_groups = 0;
    // the range opened by spinsim_range_begin, until spinsim_range_finish
    // (any other call on the handle closes it: they share the arena)
    bool range_open = false;
    spinsim_request range_req{};
    spinsim_result* range_res = nullptr;
    Plan range_plan;
    std::vector<Checked> range_checked;
    // device memory the handle holds (arena + serving pool), never above budget
    size_t held = 0, peak_held = 0;
    // host-side fault injection (SPINSIM_FAIL_ALLOC / SPINSIM_FAIL_LAUNCH at
    // spinsim_create): the n-th device allocation or kernel launch of the
    // handle reports failure instead of being made; 0 = off
    int64_t fail_alloc_at = 0, fail_launch_at = 0;
    int64_t allocs = 0, launches = 0;
    // serving: one pool of device memory, carved into the scratch of the
    // batches in flight (first fit; free pieces by offset, coalesced)
    std::vector<Slot> slots;
    DevBuf pool;
    std::map<size_t, size_t> pool_free;   // offset -> length of the free pieces
    size_t pool_in_use = 0;
    std::deque<int64_t> pending;
    std::deque<int64_t> done_order;       // tickets in order of completion (spinsim_poll_any)
    std::unordered_map<int64_t, Ticket> tickets;
    int64_t next_ticket = 1;
    int64_t requests_in_flight = 0;
};

namespace {

// Host-side fault injection: true when this allocation (or launch) is the
// one the handle was told to fail.  Nothing is sent to the GPU for it, so the
// failure paths (E_NOMEM, E_CUDA, per-request statuses, the handle staying
// usable) can be exercised without a GPU fault.
bool inject_alloc_failure(spinsim_s* h) { return h->fail_alloc_at > 0 && ++h->allocs == h->fail_alloc_at; }
bool inject_launch_failure(spinsim_s* h) { return h->fail_launch_at > 0 && ++h->launches == h->fail_launch_at; }

// Every device buffer of a handle is its main arena or its serving pool, and
// the two together never exceed the handle's budget.
void note_held(spinsim_s* h)
{
    h->held = h->arena.buf.cap + h->pool.cap;
    h->peak_held = std::max(h->peak_held, h->held);
}

int release_device(spinsim_s* h, DevBuf& b)
{
    if (!b.p) return SPINSIM_OK;
    const cudaError_t e = cudaFree(b.p);   // synchronises the device
    b.p = nullptr;
    b.cap = 0;
    note_held(h);
    return e == cudaSuccess ? SPINSIM_OK : SPINSIM_E_CUDA;
}

// Grow buffer b (the arena or the pool) to at least `need` bytes, keeping the
// handle's total within its budget (1.5x headroom while it fits, else exact).
int ensure_device(spinsim_s* h, DevBuf& b, size_t need)
{
    if (b.cap >= need) return SPINSIM_OK;
    const size_t others = h->held - b.cap;
    if (need > h->budget || others > h->budget - need) return SPINSIM_E_NOMEM;
    size_t cap = round_up(std::max(need, b.cap + b.cap / 2), size_t(1) << 20);
    if (cap > h->budget - others) cap = need;
    int st = release_device(h, b);
    if (st != SPINSIM_OK) return st;
    if (inject_alloc_failure(h) || cudaMalloc(&b.p, cap) != cudaSuccess) {
        cudaGetLastError();
        b.p = nullptr;
        return SPINSIM_E_NOMEM;
    }
    b.cap = cap;
    note_held(h);
    return SPINSIM_OK;
}

bool serving_busy(const spinsim_s* h)
{
    for (const Slot& s : h->slots)
        if (s.busy) return true;
    return false;
}

// Free the serving pool (no batch may be in flight on it).
int release_pool(spinsim_s* h)
{
    h->pool_free.clear();
    h->pool_in_use = 0;
    return release_device(h, h->pool);
}

// Grow the main arena; when the serving pool's memory stands in the way and
// no served batch is in flight, the pool is given back first.
int ensure_arena(spinsim_s* h, size_t need)
{
    int st = ensure_device(h, h->arena.buf, need);
    if (st == SPINSIM_E_NOMEM && h->pool.p && !serving_busy(h) && need <= h->budget) {
        st = release_pool(h);
        if (st != SPINSIM_OK) return st;
        st = ensure_device(h, h->arena.buf, need);
    }
    return st;
}

int ensure_pinned(PinnedBuf& b, size_t need)
{
    if (b.cap >= need) return SPINSIM_OK;
    if (b.p) cudaFreeHost(b.p);
    b.p = nullptr;
    b.cap = 0;
    size_t cap = round_up(std::max<size_t>(need, 4096), 4096);
    if (cudaMallocHost(&b.p, cap) != cudaSuccess) {
        cudaGetLastError();
        return SPINSIM_E_NOMEM;
    }
    b.cap = cap;
    return SPINSIM_OK;
}

// Parameter table of one spin group: the simulations, their sample offsets
// and their first chain-tree node per level, contiguous (uploaded with one copy).
size_t table_bytes(int64_t n, int levels)
{
    return round_up((size_t)n * sizeof(DevSim), 256) + round_up((size_t)(n + 1) * sizeof(int64_t), 256) +
           round_up((size_t)levels * (n + 1) * sizeof(int64_t), 256);
}

// Scratch bytes of one group (spin) of a batch.
// The phasor tables of `entries` entries: FP64 (re, im) pairs.
size_t phase_bytes(int64_t entries) { return round_up((size_t)entries * 2 * sizeof(double), 256); }

size_t group_bytes(int spin_x2, int64_t n, int64_t samples, const int64_t* nodes, int levels, int64_t phase_n)
{
    const size_t opb = (size_t)op_doubles(spin_x2) * sizeof(double);
    return table_bytes(n, levels) + 256 /* tile counter */ + round_up((size_t)samples * opb, 256) +
           phase_bytes(phase_n) + chain_layout(spin_x2, nodes, levels).bytes;
}

// Where the kernels can write an output: 16-byte aligned device memory as it
// is; with `direct_host`, 16-byte aligned host memory the device can address
// (pinned and mapped) through its device address; else nullptr, and the
// output is staged through the batch's scratch and copied back.  While a
// stream is being captured pointer kinds cannot be queried; outputs are then
// taken to be device memory.  *host_direct tells whether the address found
// is host memory.
double* device_view(double* p, bool capturing, bool direct_host, bool* host_direct = nullptr)
{
    if (host_direct) *host_direct = false;
    if (!p || ((uintptr_t)p & 15u) != 0) return nullptr;
    if (capturing) return p;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return p;
    if (direct_host && at.type == cudaMemoryTypeHost && at.devicePointer &&
        ((uintptr_t)at.devicePointer & 15u) == 0) {
        if (host_direct) *host_direct = true;
        return static_cast<double*>(at.devicePointer);
    }
    return nullptr;
}

bool needs_stage(double* p, bool capturing, bool direct_host)
{
    return p && !device_view(p, capturing, direct_host);
}

// Staging bytes of one request's outputs (each piece 256-byte aligned).
size_t staging_bytes(const spinsim_request& r, const spinsim_result& res, int64_t K, bool capturing, bool direct_host)
{
    const size_t N = (size_t)r.spin_x2 + 1;
    size_t b = 0;
    if (needs_stage(res.states, capturing, direct_host)) b += round_up((size_t)K * 2 * N * sizeof(double), 256);
    if (needs_stage(res.spin, capturing, direct_host)) b += round_up((size_t)K * 3 * sizeof(double), 256);
    if (needs_stage(res.ops, capturing, direct_host)) b += round_up((size_t)K * 2 * N * N * sizeof(double), 256);
    return b;
}

// Device scratch of a batch, accumulated request by request: one group per
// (spin, kernel variant) as build_plan forms them, plus the staged outputs.
// total() is the plan.total build_plan gives the same batch.
struct Footprint {
    int precision;
    int64_t count[kMaxGroups] = {}, samples[kMaxGroups] = {}, phase[kMaxGroups] = {};
    int64_t nodes[kMaxGroups][kMaxLevels] = {};
    int levels[kMaxGroups];
    size_t staged = 0;
    explicit Footprint(int prec) : precision(prec)
    {
        for (int& l : levels) l = 1;
    }
    void add(int spin_x2, int variant, int64_t K, int n_tones, size_t staged_bytes)
    {
        const int g = (spin_x2 - 1) * kVariants + variant;
        count[g] += 1;
        samples[g] += variant_pairs(spin_x2, precision, variant) ? pair_slots(K) : K;
        phase[g] += phasor_entries(K, n_tones);
        const ChainGeom cg = chain_geom(K);
        levels[g] = std::max(levels[g], cg.top + 1);
        for (int l = 0; l <= cg.top; l++) nodes[g][l] += cg.nodes[l];
        staged += staged_bytes;
    }
    size_t total() const
    {
        size_t t = staged;
        for (int g = 0; g < kMaxGroups; g++)
            if (count[g]) t += group_bytes(1 + g / kVariants, count[g], samples[g], nodes[g], levels[g], phase[g]);
        return std::max<size_t>(t, 256);
    }
};

// Build the plan: offsets inside one arena, the staged outputs, and fill the
// pinned parameter table.  `checked` holds the validation of every request.
// While a stream is being captured the pointer kinds cannot be queried; the
// outputs are then taken to be device memory (only alignment is checked).
int build_plan(const spinsim_request* reqs, spinsim_result* res, int64_t n, const std::vector<Checked>& checked,
               int precision, bool capturing, Plan& plan, bool direct_host = false)
{
    plan = Plan();
    plan.staged_of.assign((size_t)n, -1);
    plan.dev_states.assign((size_t)n, nullptr);
    plan.dev_spin.assign((size_t)n, nullptr);
    plan.dev_ops.assign((size_t)n, nullptr);
    size_t off = 0;
    size_t pin = 0;
    // one launch group per (spin, kernel variant): every request runs the
    // variant it needs on its own, so its result never depends on the batch
    for (int gi = 0; gi < kMaxGroups; gi++) {
        const int spin = 1 + gi / kVariants, variant = gi % kVariants;
        Group g;
        g.spin_x2 = spin;
        g.variant = variant;
        for (int64_t i = 0; i < n; i++)
            if (checked[i].status == SPINSIM_OK && reqs[i].spin_x2 == spin && checked[i].variant == variant) {
                g.idx.push_back(i);
                g.samples += variant_pairs(spin, precision, variant) ? pair_slots(checked[i].K) : checked[i].K;
                g.phase_n += phasor_entries(checked[i].K, reqs[i].field.n_tones);
                g.steps += (double)checked[i].K * (double)checked[i].L;
                g.min_seg_log2 = std::min(g.min_seg_log2, seg_log2_of(checked[i].L));
                const ChainGeom cg = chain_geom(checked[i].K);
                g.levels = std::max(g.levels, cg.top + 1);
                g.max_run = std::max(g.max_run, cg.run);
                for (int l = 0; l <= cg.top; l++) g.nodes[l] += cg.nodes[l];
            }
        if (g.idx.empty()) continue;
        const int64_t m = (int64_t)g.idx.size();
        const size_t opb = (size_t)op_doubles(spin) * sizeof(double);
        g.sims_off = off;
        g.soff_off = off + round_up((size_t)m * sizeof(DevSim), 256);
        g.loff_off = g.soff_off + round_up((size_t)(m + 1) * sizeof(int64_t), 256);
        off += table_bytes(m, g.levels);
        g.counter_off = off; off += 256;
        g.U_off = off; off += round_up((size_t)g.samples * opb, 256);
        g.phase_off = off; off += phase_bytes(g.phase_n);
        g.chain = chain_layout(spin, g.nodes, g.levels);
        g.chain_off = off; off += g.chain.bytes;
        pin += table_bytes(m, g.levels);
        plan.groups.push_back(std::move(g));
    }
    // host-resident or misaligned outputs are staged through the arena
    // (unless written directly into mapped host memory)
    for (const Group& g : plan.groups)
        for (int64_t i : g.idx) {
            const int N = reqs[i].spin_x2 + 1;
            const int64_t K = checked[i].K;
            spinsim_result& r = res[i];
            bool hs = false, hp = false, ho = false;
            plan.dev_states[i] = device_view(r.states, capturing, direct_host, &hs);
            plan.dev_spin[i] = device_view(r.spin, capturing, direct_host, &hp);
            plan.dev_ops[i] = device_view(r.ops, capturing, direct_host, &ho);
            plan.direct_host_bytes += (hs ? (size_t)K * 2 * N * sizeof(double) : 0) +
                                      (hp ? (size_t)K * 3 * sizeof(double) : 0) +
                                      (ho ? (size_t)K * 2 * N * N * sizeof(double) : 0);
            bool st = r.states && !plan.dev_states[i], sp = r.spin && !plan.dev_spin[i],
                 op = r.ops && !plan.dev_ops[i];
            if (!(st || sp || op)) continue;
            plan.staged_of[i] = (int64_t)plan.staged.size();
            StagedOut so{};
            so.req = i;
            if (st) { so.host_states = r.states; so.states_bytes = (size_t)K * 2 * N * sizeof(double); so.states_off = off; off += round_up(so.states_bytes, 256); }
            if (sp) { so.host_spin = r.spin; so.spin_bytes = (size_t)K * 3 * sizeof(double); so.spin_off = off; off += round_up(so.spin_bytes, 256); }
            if (op) { so.host_ops = r.ops; so.ops_bytes = (size_t)K * 2 * N * N * sizeof(double); so.ops_off = off; off += round_up(so.ops_bytes, 256); }
            plan.staged.push_back(so);
        }
    plan.total = std::max<size_t>(off, 256);
    plan.pinned_bytes = pin;
    return SPINSIM_OK;
}

// Fill the pinned parameter tables of every group; `base` is the arena's
// device base address the tables will refer to.
void fill_tables(spinsim_s* h, const spinsim_request* reqs, spinsim_result* res, const std::vector<Checked>& checked,
                 const Plan& plan, char* base, char* pinned)
{
    size_t pin = 0;
    for (const Group& g : plan.groups) {
        const int64_t m = (int64_t)g.idx.size();
        DevSim* sims = reinterpret_cast<DevSim*>(pinned + pin);
        int64_t* soff = reinterpret_cast<int64_t*>(pinned + pin + (g.soff_off - g.sims_off));
        int64_t* loff = reinterpret_cast<int64_t*>(pinned + pin + (g.loff_off - g.sims_off));
        pin += table_bytes(m, g.levels);
        int64_t so = 0, eo = 0;
        int64_t lo[kMaxLevels] = {};
        for (int64_t q = 0; q < m; q++) {
            const int64_t i = g.idx[q];
            const spinsim_request& r = reqs[i];
            DevSim d;
            fill_devsim(h->cfg, r, checked[i].K, checked[i].L, d);
            d.states = plan.dev_states[i];
            d.spin = plan.dev_spin[i];
            d.ops = plan.dev_ops[i];
            if (plan.staged_of[i] >= 0) {
                const StagedOut& s = plan.staged[(size_t)plan.staged_of[i]];
                if (s.host_states) d.states = reinterpret_cast<double*>(base + s.states_off);
                if (s.host_spin) d.spin = reinterpret_cast<double*>(base + s.spin_off);
                if (s.host_ops) d.ops = reinterpret_cast<double*>(base + s.ops_off);
            }
            d.sample_offset = so;
            soff[q] = so;
            so += variant_pairs(g.spin_x2, h->cfg.precision, g.variant) ? pair_slots(d.K) : d.K;
            d.eb_tab = reinterpret_cast<const double*>(base + g.phase_off) + 2 * eo;
            d.eb_off = eo;
            eo += phasor_entries(d.K, d.n_tones);
            const ChainGeom cg = chain_geom(d.K);
            d.chain_run = cg.run;
            d.chain_top = cg.top;
            for (int l = 0; l < g.levels; l++) {
                loff[(size_t)l * (m + 1) + q] = lo[l];
                lo[l] += l <= cg.top ? cg.nodes[l] : 0;
            }
            res[i].trotter_squares = d.tau;
            h->last.trotter_squares = std::max(h->last.trotter_squares, d.tau);
            d.spin_x2 = r.spin_x2;
            sims[q] = d;
        }
        soff[m] = so;
        for (int l = 0; l < g.levels; l++) loff[(size_t)l * (m + 1) + m] = lo[l];
    }
}

// Resident blocks per SM of an integrate shape; computed outside stream
// capture (it sets the kernel's shared-memory limit) and cached.
int occupancy(spinsim_s* h, int spin, int block, int variant, bool capturing, int* per_sm)
{
    auto key = std::make_tuple(spin, block, variant);
    auto it = h->occ.find(key);
    if (it != h->occ.end()) {
        *per_sm = it->second;
        return SPINSIM_OK;
    }
    if (capturing) return SPINSIM_E_UNSUPPORTED;
    int b = 0;
    if (integrate_occupancy(spin, h->cfg.precision, h->cfg.method, block, variant, &b) != cudaSuccess) {
        cudaGetLastError();
        return SPINSIM_E_CUDA;
    }
    h->occ[key] = b;
    *per_sm = b;
    return SPINSIM_OK;
}

int size_bucket(int64_t samples)
{
    int b = 0;
    while (samples > 1 && b < 60) { samples >>= 1; b++; }
    return b;
}

// Choose (lanes per sample, threads per block) for the integrate kernel and
// its resident blocks per SM.  Results never depend on this choice; only the
// time does.  Explicit configuration values are kept; lanes and block size are
// tuned by timing trial launches, once per (device, key), and cached.  The
// resident blocks per SM are the explicit value or the most the kernel allows
// (fewer never paid on GB300: the tail they save costs more in issue rate).
int choose_shape(spinsim_s* h, int spin, int variant, double steps, int min_seg_log2, IntegrateArgs& a,
                 cudaStream_t stream, bool capturing, int& lanes, int& block, int& grid)
{
    const int precision = h->cfg.precision;
    const int method = h->cfg.method;
    const int per_slot = variant_pairs(spin, precision, variant) ? 2 : 1;   // samples per lane group
    lanes = h->cfg.lanes_per_sample;
    block = h->cfg.threads_per_block;
    int bps = h->cfg.blocks_per_sm;
    const bool full_trial = steps <= kFullTrialSteps;
    if (lanes == 0 || block == 0) {
        TuneKey key{spin, precision, method, h->tau, variant, (int64_t)size_bucket(a.total_samples) * 8 + min_seg_log2};
        bool found = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find({h->device, key});
            if (it != g_tune_cache.end()) {
                if (lanes == 0) lanes = it->second.lanes;
                if (block == 0) block = it->second.block;
                found = true;
            }
        }
        if (!found) {
            // bulk tiles: one lane per sample unless configured (with the
            // per-tile epilogue more lanes per sample never paid on GB300;
            // the samples after the last whole wave use more anyway)
            const int lane_opts[1] = {1};
            const int block_opts[3] = {64, 128, 256};
            int best_l = lanes ? lanes : 1, best_b = block ? block : 128;
            if (!capturing) {
                float best = 1e30f;
                float trial_per[3] = {1e30f, 1e30f, 1e30f};   // per block_opts entry
                cudaEvent_t e0, e1;
                if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SPINSIM_E_CUDA;
                for (int li = 0; li < 1; li++) {
                    const int L = lanes ? lanes : lane_opts[li];
                    if (lanes && li > 0) break;
                    if (!lanes && L > (1 << min_seg_log2)) break;   // no more lanes than segments
                    for (int bi = 0; bi < 3; bi++) {
                        const int B = block ? block : block_opts[bi];
                        if (block && bi > 0) break;
                        int per_sm = 0;
                        if (occupancy(h, spin, B, variant, false, &per_sm) != SPINSIM_OK || per_sm < 1) continue;
                        const int P = bps ? std::min(bps, per_sm) : per_sm;
                        const int64_t wave_blocks = (int64_t)h->n_sm * P;
                        IntegrateArgs t = a;
                        if (!full_trial) {
                            // a prefix of at most 4 full waves of this shape
                            t.total_samples = std::min<int64_t>(a.total_samples, 4 * wave_blocks * (B / L) * per_slot);
                        }
                        integrate_tiles(t.total_samples, L, B, wave_blocks, min_seg_log2, t, per_slot);
                        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((t.n_tiles + B / 32 - 1) / (B / 32), wave_blocks));
                        float ms_best = 1e30f;
                        for (int rep = 0; rep < 2; rep++) {
                            cudaMemsetAsync(a.tile_counter, 0, sizeof(unsigned long long), stream);
                            cudaEventRecord(e0, stream);
                            launch_integrate(spin, precision, method, B, g, variant, t, stream);
                            cudaEventRecord(e1, stream);
                            if (cudaEventSynchronize(e1) != cudaSuccess) {
                                cudaEventDestroy(e0);
                                cudaEventDestroy(e1);
                                return SPINSIM_E_CUDA;
                            }
                            float ms = 0.f;
                            cudaEventElapsedTime(&ms, e0, e1);
                            ms_best = std::min(ms_best, ms);
                        }
                        const float per = ms_best / (float)std::max<int64_t>(1, t.total_samples);
                        trial_per[bi] = per;
                        if (per < best) {
                            best = per;
                            best_l = L;
                            best_b = B;
                        }
                    }
                }
                // the largest block within 2 % of the best trial: the trials time
                // a prefix of a few waves, where the shapes come out within their
                // noise, while over a whole large batch one block of eight warps
                // per SM measured fastest (the 4096-simulation sweep: 151.0 ms
                // with 256 threads, 153.4 ms with 64 or 128)
                if (!block)
                    for (int bi = 2; bi >= 0; bi--)
                        if (trial_per[bi] <= best * 1.02f) {
                            best_b = block_opts[bi];
                            break;
                        }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                std::lock_guard<std::mutex> lk(g_tune_mu);
                g_tune_cache[{h->device, key}] = TuneVal{best_l, best_b};
            }
            lanes = best_l;
            block = best_b;
        }
    }
    int per_sm = 0;
    int st = occupancy(h, spin, block, variant, capturing, &per_sm);
    if (st != SPINSIM_OK) return st;
    per_sm = std::max(per_sm, 1);
    if (bps > 0) per_sm = std::min(per_sm, bps);
    const int64_t wave_blocks = (int64_t)h->n_sm * per_sm;
    integrate_tiles(a.total_samples, lanes, block, wave_blocks, min_seg_log2, a, per_slot);
    grid = (int)std::max<int64_t>(1, std::min<int64_t>((a.n_tiles + block / 32 - 1) / (block / 32), wave_blocks));
    return SPINSIM_OK;
}

// Write the parameter tables of `plan` into the pinned buffer.  The buffer
// may still be read by an earlier, not yet executed, host-to-device copy: when
// the content is unchanged nothing is written (and nothing waited for);
// otherwise the earlier copy is waited for through `pinned_free`.
int refresh_table(spinsim_s* h, const spinsim_request* reqs, spinsim_result* res, const std::vector<Checked>& checked,
                  const Plan& plan, char* base, PinnedBuf& pinned, cudaEvent_t pinned_free, bool capturing)
{
    if (h->table_tmp.size() < plan.pinned_bytes) h->table_tmp.resize(plan.pinned_bytes);
    fill_tables(h, reqs, res, checked, plan, base, h->table_tmp.data());
    if (plan.pinned_bytes <= pinned.cap && std::memcmp(pinned.p, h->table_tmp.data(), plan.pinned_bytes) == 0)
        return SPINSIM_OK;
    if (pinned_free && cudaEventSynchronize(pinned_free) != cudaSuccess) return SPINSIM_E_CUDA;
    if (plan.pinned_bytes > pinned.cap) {
        if (capturing) return SPINSIM_E_UNSUPPORTED;
        int st = ensure_pinned(pinned, plan.pinned_bytes);
        if (st != SPINSIM_OK) return st;
    }
    std::memcpy(pinned.p, h->table_tmp.data(), plan.pinned_bytes);
    return SPINSIM_OK;
}

// Enqueue one batch on `stream` using `arena` and the pinned table buffer.
// Requests with a failed validation are skipped.
// With `prof_in_graph`, a capture of the handle's own graph records the
// profiling events as event nodes, so every replay times its kernels.
// `phase`: kPhaseAll the whole path; kPhaseBegin the operators and the chain's
// up-sweeps only (spinsim_range_begin); kPhaseFinish the chain's down-sweeps
// and the write from each request's psi0, over operators a kPhaseBegin run of
// the same plan left in the arena (spinsim_range_finish).
enum { kPhaseAll = 0, kPhaseBegin = 1, kPhaseFinish = 2 };

int run_batch(spinsim_s* h, const spinsim_request* reqs, spinsim_result* res, const std::vector<Checked>& checked,
              const Plan& plan, cudaStream_t stream, Arena& arena, PinnedBuf& pinned, cudaEvent_t pinned_free,
              bool capturing, int* kernels_out, bool prof_in_graph = false, int phase = kPhaseAll)
{
    auto prof_record = [&](cudaEvent_t e) {
        if (capturing) cudaEventRecordWithFlags(e, stream, cudaEventRecordExternal);
        else cudaEventRecord(e, stream);
    };
    if (plan.groups.empty()) {
        if (kernels_out) *kernels_out = 0;
        return SPINSIM_OK;
    }
    if (plan.total > arena.buf.cap) {
        // only the handle's own arena grows here; a serving batch's piece of
        // the pool is carved at its plan's size
        if (capturing || &arena != &h->arena) return SPINSIM_E_UNSUPPORTED;
        int st = ensure_arena(h, plan.total);
        if (st != SPINSIM_OK) return st;
    }
    char* base = static_cast<char*>(arena.buf.p);
    int st = refresh_table(h, reqs, res, checked, plan, base, pinned, pinned_free, capturing);
    if (st != SPINSIM_OK) return st;
    int kernels = 0;
    size_t pin = 0;
    for (const Group& g : plan.groups) {
        const int64_t m = (int64_t)g.idx.size();
        const size_t tbl = table_bytes(m, g.levels);
        // the table is contiguous in both the pinned buffer and the arena
        if (cudaMemcpyAsync(base + g.sims_off, static_cast<char*>(pinned.p) + pin, tbl, cudaMemcpyHostToDevice,
                            stream) != cudaSuccess)
            return SPINSIM_E_CUDA;
        pin += tbl;
        h->last.h2d_bytes += (int64_t)tbl;
        const int pg = (h->cfg.profile && (!capturing || prof_in_graph) && h->prof_groups < kMaxGroups)
                           ? h->prof_groups++
                           : -1;
        if (pinned_free && cudaEventRecord(pinned_free, stream) != cudaSuccess) return SPINSIM_E_CUDA;
        IntegrateArgs ia;
        ia.sims = reinterpret_cast<const DevSim*>(base + g.sims_off);
        ia.sample_offsets = reinterpret_cast<const int64_t*>(base + g.soff_off);
        ia.n_sims = (int)m;
        ia.total_samples = g.samples;
        ia.U = reinterpret_cast<double*>(base + g.U_off);
        ia.tau = h->tau;
        ia.tile_counter = reinterpret_cast<unsigned long long*>(base + g.counter_off);
        int lanes = 0, block = 0, grid = 0;
        if (g.samples > 0) {
            if (phase == kPhaseFinish && pg >= 0) prof_record(h->prof[pg][0]);
            if (phase != kPhaseFinish) {
                st = choose_shape(h, g.spin_x2, g.variant, g.steps, g.min_seg_log2, ia, stream, capturing, lanes, block,
                                  grid);
                if (st != SPINSIM_OK) return st;
                if (cudaMemsetAsync(ia.tile_counter, 0, sizeof(unsigned long long), stream) != cudaSuccess)
                    return SPINSIM_E_CUDA;
                // the integrate time includes the drive phasor tables' kernel,
                // which it overlaps (nothing may stand between the two launches)
                if (pg >= 0) prof_record(h->prof[pg][0]);
                if (g.phase_n > 0) {
                    if (inject_launch_failure(h) ||
                        launch_phase_table(ia.sims, (int)m, g.phase_n, reinterpret_cast<double*>(base + g.phase_off),
                                           h->n_sm, stream) != cudaSuccess)
                        return SPINSIM_E_CUDA;
                    kernels += 1;
                }
                if (inject_launch_failure(h) ||
                    launch_integrate(g.spin_x2, h->cfg.precision, h->cfg.method, block, grid, g.variant, ia, stream,
                                     g.phase_n > 0) !=
                        cudaSuccess)
                    return SPINSIM_E_CUDA;
                kernels += 1;
            }
            if (pg >= 0) prof_record(h->prof[pg][1]);
            ChainArgs ca;
            ca.sims = ia.sims;
            ca.n_sims = (int)m;
            ca.level_off = reinterpret_cast<const int64_t*>(base + g.loff_off);
            ca.U = ia.U;
            chain_args_set(ca, g.chain, base + g.chain_off);
            ca.max_run = g.max_run;
            ca.mode = phase == kPhaseBegin ? kChainUp : (phase == kPhaseFinish ? kChainDown : kChainFull);
            int chain_k = 0;
            if (inject_launch_failure(h) ||
                launch_chain(g.spin_x2, ca, h->n_sm, stream, &chain_k, h->cfg.chain_precision == 1) != cudaSuccess)
                return SPINSIM_E_CUDA;
            if (pg >= 0) prof_record(h->prof[pg][2]);
            kernels += chain_k;
            h->last.lanes_per_sample = lanes;
            h->last.threads_per_block = block;
            h->last.grid_blocks = grid;
        }
    }
    if (phase == kPhaseBegin) {
        if (kernels_out) *kernels_out = kernels;
        return SPINSIM_OK;
    }
    for (const StagedOut& s : plan.staged)
        h->last.d2h_bytes += (int64_t)((s.host_states ? s.states_bytes : 0) + (s.host_spin ? s.spin_bytes : 0) +
                                       (s.host_ops ? s.ops_bytes : 0));
    h->last.d2h_bytes += (int64_t)plan.direct_host_bytes;
    for (const StagedOut& s : plan.staged) {
        if (s.host_states && cudaMemcpyAsync(s.host_states, base + s.states_off, s.states_bytes, cudaMemcpyDefault, stream) != cudaSuccess)
            return SPINSIM_E_CUDA;
        if (s.host_spin && cudaMemcpyAsync(s.host_spin, base + s.spin_off, s.spin_bytes, cudaMemcpyDefault, stream) != cudaSuccess)
            return SPINSIM_E_CUDA;
        if (s.host_ops && cudaMemcpyAsync(s.host_ops, base + s.ops_off, s.ops_bytes, cudaMemcpyDefault, stream) != cudaSuccess)
            return SPINSIM_E_CUDA;
    }
    if (kernels_out) *kernels_out = kernels;
    return SPINSIM_OK;
}

// Signature of a batch for graph reuse: everything except field values.
std::vector<uint64_t> batch_signature(const spinsim_request* reqs, const spinsim_result* res, int64_t n,
                                      const std::vector<Checked>& checked)
{
    std::vector<uint64_t> s;
    s.reserve((size_t)n * 6 + 1);
    s.push_back((uint64_t)n);
    for (int64_t i = 0; i < n; i++) {
        s.push_back((uint64_t)reqs[i].spin_x2 | ((uint64_t)(checked[i].status & 0xff) << 8) |
                    ((uint64_t)checked[i].variant << 16));
        s.push_back((uint64_t)checked[i].K);
        s.push_back((uint64_t)checked[i].L);
        s.push_back((uint64_t)(uintptr_t)res[i].states);
        s.push_back((uint64_t)(uintptr_t)res[i].spin);
        s.push_back((uint64_t)(uintptr_t)res[i].ops);
    }
    return s;
}

void drop_graph(spinsim_s* h)
{
    if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
    h->graph_exec = nullptr;
    h->graph_sig.clear();
    h->graph_prof_groups = 0;
    h->memo_reqs.clear();
    h->memo_res.clear();
}

// True when (reqs, res) repeat the call remembered with the handle's graph:
// the same requests byte for byte and the same result buffers.
bool repeats_memo(const spinsim_s* h, const spinsim_request* reqs, const spinsim_result* res, int64_t n)
{
    if (!h->graph_exec || (int64_t)h->memo_reqs.size() != n || n == 0) return false;
    if (std::memcmp(reqs, h->memo_reqs.data(), (size_t)n * sizeof(spinsim_request)) != 0) return false;
    for (int64_t i = 0; i < n; i++) {
        const spinsim_result& a = res[i];
        const spinsim_result& b = h->memo_res[i];
        if (a.states != b.states || a.spin != b.spin || a.ops != b.ops || a.capacity != b.capacity) return false;
    }
    return true;
}

void remember(spinsim_s* h, const spinsim_request* reqs, const spinsim_result* res, int64_t n)
{
    h->memo_reqs.assign(reqs, reqs + n);
    h->memo_res.assign(res, res + n);
}

}  // namespace

// ===================================================================== ABI
extern "C" {

const char* spinsim_status_string(int status)
{
    switch (status) {
        case SPINSIM_OK: return "ok";
        case SPINSIM_PENDING: return "pending";
        case SPINSIM_E_ARG: return "invalid argument";
        case SPINSIM_E_STEP_RATIO: return "time span, output step and integration step are not integer ratios";
        case SPINSIM_E_NORM: return "initial state is not normalised";
        case SPINSIM_E_NOMEM: return "device memory budget exceeded or allocation failed";
        case SPINSIM_E_CUDA: return "CUDA runtime error";
        case SPINSIM_E_TIMEOUT: return "timed out";
        case SPINSIM_E_CAPACITY: return "result capacity smaller than the number of samples";
        case SPINSIM_E_UNSUPPORTED: return "unsupported";
        default: return "unknown status";
    }
}

int spinsim_config_default(spinsim_config* cfg)
{
    if (!cfg) return SPINSIM_E_ARG;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->method = SPINSIM_METHOD_CF4;
    cfg->precision = SPINSIM_PREC_FP32_BULK;
    cfg->rotating_frame = 1;
    cfg->trotter_squares = -1;
    cfg->direct_host_outputs = 1;
    return SPINSIM_OK;
}

int spinsim_create(const spinsim_config* cfg, spinsim_handle* out)
{
    if (!cfg || !out) return SPINSIM_E_ARG;
    *out = nullptr;
    if (cfg->method < 0 || cfg->method > 2 || cfg->precision < 0 || cfg->precision > 1 ||
        cfg->trotter_squares < -1 || cfg->trotter_squares > 40 ||
        !(cfg->lanes_per_sample == 0 || cfg->lanes_per_sample == 1 || cfg->lanes_per_sample == 2 ||
          cfg->lanes_per_sample == 4 || cfg->lanes_per_sample == 8) ||
        !(cfg->threads_per_block == 0 || cfg->threads_per_block == 64 || cfg->threads_per_block == 128 ||
          cfg->threads_per_block == 256) ||
        cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 32 || cfg->mem_budget < 0 || cfg->chain_precision < 0 ||
        cfg->chain_precision > 1 || cfg->direct_host_outputs < 0 || cfg->direct_host_outputs > 1)
        return SPINSIM_E_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg->device < 0 || cfg->device >= ndev) {
        cudaGetLastError();
        return SPINSIM_E_CUDA;
    }
    if (cudaSetDevice(cfg->device) != cudaSuccess) return SPINSIM_E_CUDA;
    spinsim_s* h = new (std::nothrow) spinsim_s();
    if (!h) return SPINSIM_E_NOMEM;
    h->cfg = *cfg;
    h->device = cfg->device;
    h->tau = cfg->trotter_squares;   // -1: chosen per request (choose_tau)
    cudaDeviceGetAttribute(&h->n_sm, cudaDevAttrMultiProcessorCount, cfg->device);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        delete h;
        return SPINSIM_E_CUDA;
    }
    h->budget = cfg->mem_budget > 0 ? (size_t)cfg->mem_budget : (size_t)(0.9 * (double)free_b);
    auto env_count = [](const char* name) -> int64_t {
        const char* v = std::getenv(name);
        if (!v || !*v) return 0;
        char* end = nullptr;
        const long long n = std::strtoll(v, &end, 10);
        return (end && *end == '\0' && n > 0) ? (int64_t)n : 0;
    };
    h->fail_alloc_at = env_count("SPINSIM_FAIL_ALLOC");
    h->fail_launch_at = env_count("SPINSIM_FAIL_LAUNCH");
    if (cudaStreamCreateWithFlags(&h->work, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_pinned, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_done, cudaEventDisableTiming) != cudaSuccess) {
        spinsim_destroy(h);
        return SPINSIM_E_CUDA;
    }
    if (cfg->profile)
        for (auto& row : h->prof)
            for (auto& e : row)
                if (cudaEventCreate(&e) != cudaSuccess) {
                    spinsim_destroy(h);
                    return SPINSIM_E_CUDA;
                }
    *out = h;
    return SPINSIM_OK;
}

void spinsim_destroy(spinsim_handle h)
{
    if (!h) return;
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    drop_graph(h);
    for (Slot& s : h->slots) {
        if (s.pinned.p) cudaFreeHost(s.pinned.p);
        if (s.done) cudaEventDestroy(s.done);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (h->arena.buf.p) cudaFree(h->arena.buf.p);
    if (h->pool.p) cudaFree(h->pool.p);
    if (h->pinned.p) cudaFreeHost(h->pinned.p);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    if (h->ev_out) cudaEventDestroy(h->ev_out);
    if (h->ev_pinned) cudaEventDestroy(h->ev_pinned);
    if (h->ev_done) cudaEventDestroy(h->ev_done);
    for (auto& row : h->prof)
        for (auto& e : row)
            if (e) cudaEventDestroy(e);
    if (h->work) cudaStreamDestroy(h->work);
    delete h;
}

int spinsim_counts(const spinsim_request* req, int64_t* K, int64_t* L)
{
    Checked c = check_request(req);
    if (c.status != SPINSIM_OK) return c.status;
    if (K) *K = c.K;
    if (L) *L = c.L;
    return SPINSIM_OK;
}

int64_t spinsim_footprint(spinsim_handle h, const spinsim_request* reqs, int64_t n)
{
    if (!h || (n > 0 && !reqs) || n < 0) return SPINSIM_E_ARG;
    Footprint fp(h->cfg.precision);
    for (int64_t i = 0; i < n; i++) {
        Checked c = check_request(&reqs[i]);
        if (c.status != SPINSIM_OK) return c.status;
        fp.add(reqs[i].spin_x2, request_variant(h->cfg, reqs[i], c.K, c.L), c.K, reqs[i].field.n_tones, 0);
    }
    return n > 0 ? (int64_t)fp.total() : 0;
}

int spinsim_simulate(spinsim_handle h, const spinsim_request* reqs, spinsim_result* res, int64_t n, void* stream_v)
{
    if (!h || n < 0 || (n > 0 && (!reqs || !res))) return SPINSIM_E_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return SPINSIM_E_CUDA;
    h->range_open = false;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    if (h->cfg.use_graphs && repeats_memo(h, reqs, res, n)) {
        // the same batch again: its parameter table is the one in the pinned
        // buffer; replay the graph (table upload, kernels, copies) as it is
        cudaStreamCaptureStatus cap0 = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(stream, &cap0) == cudaSuccess && cap0 == cudaStreamCaptureStatusNone) {
            for (int64_t i = 0; i < n; i++) {
                res[i].status = h->memo_res[i].status;
                res[i].flags = h->memo_res[i].flags;
                res[i].n_samples = h->memo_res[i].n_samples;
                res[i].trotter_squares = h->memo_res[i].trotter_squares;
            }
            if (h->done_pending && cudaStreamWaitEvent(stream, h->ev_done, 0) != cudaSuccess) return SPINSIM_E_CUDA;
            if (cudaGraphLaunch(h->graph_exec, stream) != cudaSuccess) return SPINSIM_E_CUDA;
            if (cudaEventRecord(h->ev_pinned, stream) != cudaSuccess || cudaEventRecord(h->ev_done, stream) != cudaSuccess)
                return SPINSIM_E_CUDA;
            h->done_pending = true;
            h->last = h->graph_info;
            h->last.graph_replayed = 1;
            h->last.integrate_ms = -1.0;
            h->last.chain_ms = -1.0;
            h->prof_groups = h->graph_prof_groups;
            h->last.kernels_launched = h->graph_kernels;
            int first = SPINSIM_OK;
            for (int64_t i = 0; i < n && first == SPINSIM_OK; i++) first = res[i].status;
            return first;
        }
        cudaGetLastError();
    }
    std::vector<Checked> checked((size_t)n);
    int first_err = SPINSIM_OK;
    for (int64_t i = 0; i < n; i++) {
        checked[i] = check_request(&reqs[i]);
        if (checked[i].status == SPINSIM_OK) checked[i].status = precision_status(h->cfg, reqs[i]);
        if (checked[i].status == SPINSIM_OK) {
            if (!res[i].states) checked[i].status = SPINSIM_E_ARG;
            else if (res[i].capacity < checked[i].K) checked[i].status = SPINSIM_E_CAPACITY;
        }
        res[i].status = checked[i].status;
        if (checked[i].status == SPINSIM_OK) {
            checked[i].flags |= precision_flags(h->cfg.precision, h->cfg.rotating_frame, reqs[i]);
            checked[i].variant = request_variant(h->cfg, reqs[i], checked[i].K, checked[i].L);
        }
        res[i].flags = checked[i].flags;
        res[i].trotter_squares = 0;
        res[i].n_samples = checked[i].status == SPINSIM_OK ? checked[i].K : 0;
        if (checked[i].status != SPINSIM_OK && first_err == SPINSIM_OK) first_err = checked[i].status;
    }
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusNone;
    }
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    // a batch that cannot run: every request that was to run carries the error
    auto fail = [&](int e) {
        for (int64_t i = 0; i < n; i++)
            if (checked[i].status == SPINSIM_OK) {
                res[i].status = e;
                res[i].n_samples = 0;
            }
        return e;
    };
    h->last = spinsim_launch_info{};
    h->last.trotter_squares = 0;
    h->last.integrate_ms = -1.0;
    h->last.chain_ms = -1.0;
    h->prof_groups = 0;
    int kernels = 0;
    int st = SPINSIM_OK;
    if (h->cfg.use_graphs && !capturing) {
        // A new batch shape runs eagerly on the internal stream (joined to the
        // caller's stream by events) and is captured there as a graph; later
        // calls of the same shape replay the graph on the caller's stream.
        std::vector<uint64_t> sig = batch_signature(reqs, res, n, checked);
        Plan plan;
        build_plan(reqs, res, n, checked, h->cfg.precision, false, plan, h->cfg.direct_host_outputs != 0);
        if (h->graph_exec && sig == h->graph_sig) {
            // same shape: refresh the pinned parameter table and replay on the
            // caller's stream (after the handle's previous replay)
            st = refresh_table(h, reqs, res, checked, plan, static_cast<char*>(h->arena.buf.p), h->pinned,
                               h->ev_pinned, false);
            if (st != SPINSIM_OK) return fail(st);
            if (h->done_pending && cudaStreamWaitEvent(stream, h->ev_done, 0) != cudaSuccess) return fail(SPINSIM_E_CUDA);
            if (cudaGraphLaunch(h->graph_exec, stream) != cudaSuccess) return fail(SPINSIM_E_CUDA);
            if (cudaEventRecord(h->ev_pinned, stream) != cudaSuccess || cudaEventRecord(h->ev_done, stream) != cudaSuccess)
                return fail(SPINSIM_E_CUDA);
            h->done_pending = true;
            h->last = h->graph_info;
            h->last.graph_replayed = 1;
            h->last.integrate_ms = -1.0;
            h->last.chain_ms = -1.0;
            h->prof_groups = h->graph_prof_groups;   // the replay recorded these events
            kernels = h->graph_kernels;
        } else {
            drop_graph(h);
            // on the internal stream, after the caller's earlier work and the
            // handle's last replay
            if (cudaEventRecord(h->ev_in, stream) != cudaSuccess || cudaStreamWaitEvent(h->work, h->ev_in, 0) != cudaSuccess)
                return fail(SPINSIM_E_CUDA);
            if (h->done_pending && cudaStreamWaitEvent(h->work, h->ev_done, 0) != cudaSuccess) return fail(SPINSIM_E_CUDA);
            // first run eagerly: sizes scratch and tunes the launch shape
            st = run_batch(h, reqs, res, checked, plan, h->work, h->arena, h->pinned, h->ev_pinned, false, &kernels);
            if (st != SPINSIM_OK) return fail(st);
            if (cudaStreamSynchronize(h->work) != cudaSuccess) return fail(SPINSIM_E_CUDA);
            // then capture the same batch for later replays
            // (the eager run's profiling events keep their timestamps: recording
            // them as graph nodes during the capture does not touch them)
            cudaGraph_t graph = nullptr;
            const int eager_prof = h->prof_groups;
            const spinsim_launch_info eager_info = h->last;   // the capture must not count its copies twice
            h->prof_groups = 0;
            if (cudaStreamBeginCapture(h->work, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                int k2 = 0;
                int st2 = run_batch(h, reqs, res, checked, plan, h->work, h->arena, h->pinned, nullptr, true, &k2,
                                    true);
                cudaError_t ec = cudaStreamEndCapture(h->work, &graph);
                if (st2 == SPINSIM_OK && ec == cudaSuccess && graph) {
                    if (cudaGraphInstantiate(&h->graph_exec, graph, 0) == cudaSuccess) {
                        h->graph_sig = sig;
                        h->graph_kernels = k2;
                        h->graph_prof_groups = h->prof_groups;
                        h->graph_info = eager_info;
                    } else {
                        h->graph_exec = nullptr;
                    }
                }
                if (graph) cudaGraphDestroy(graph);
                cudaGetLastError();
            } else {
                cudaGetLastError();
            }
            h->prof_groups = eager_prof;
            h->last = eager_info;
            cudaEventRecord(h->ev_pinned, h->work);
            if (cudaEventRecord(h->ev_out, h->work) != cudaSuccess || cudaStreamWaitEvent(stream, h->ev_out, 0) != cudaSuccess ||
                cudaEventRecord(h->ev_done, h->work) != cudaSuccess)
                return fail(SPINSIM_E_CUDA);
            h->done_pending = true;
        }
    } else {
        Plan plan;
        build_plan(reqs, res, n, checked, h->cfg.precision, capturing, plan, h->cfg.direct_host_outputs != 0);
        st = run_batch(h, reqs, res, checked, plan, stream, h->arena, h->pinned, capturing ? nullptr : h->ev_pinned,
                       capturing, &kernels);
        if (st != SPINSIM_OK) return fail(st);
    }
    h->last.kernels_launched = kernels;
    if (cudaGetLastError() != cudaSuccess) return fail(SPINSIM_E_CUDA);
    if (h->cfg.use_graphs && !capturing && h->graph_exec) remember(h, reqs, res, n);   // this call's graph
    return first_err;
}

int spinsim_range_begin(spinsim_handle h, const spinsim_request* req, spinsim_result* res, double* agg,
                        void* stream_v)
{
    if (!h || !req || !res || !agg) return SPINSIM_E_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return SPINSIM_E_CUDA;
    h->range_open = false;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    std::vector<Checked> checked(1);
    checked[0] = check_request(req);
    if (checked[0].status == SPINSIM_OK) checked[0].status = precision_status(h->cfg, *req);
    Checked& c = checked[0];
    if (c.status == SPINSIM_OK) {
        if (!res->states) c.status = SPINSIM_E_ARG;
        else if (res->capacity < c.K) c.status = SPINSIM_E_CAPACITY;
    }
    if (c.status == SPINSIM_OK) {
        c.flags |= precision_flags(h->cfg.precision, h->cfg.rotating_frame, *req);
        c.variant = request_variant(h->cfg, *req, c.K, c.L);
    }
    res->status = c.status;
    res->flags = c.flags;
    res->trotter_squares = 0;
    res->n_samples = 0;
    if (c.status != SPINSIM_OK) return c.status;
    // the arena is shared with graph replays: start after the handle's last
    // one, and do not replay a graph over the range's operators later
    if (h->done_pending && cudaStreamWaitEvent(stream, h->ev_done, 0) != cudaSuccess) return SPINSIM_E_CUDA;
    drop_graph(h);
    h->last = spinsim_launch_info{};
    h->last.integrate_ms = -1.0;
    h->last.chain_ms = -1.0;
    h->prof_groups = 0;
    Plan plan;
    build_plan(req, res, 1, checked, h->cfg.precision, false, plan, h->cfg.direct_host_outputs != 0);
    int kernels = 0;
    int st = run_batch(h, req, res, checked, plan, stream, h->arena, h->pinned, h->ev_pinned, false, &kernels, false,
                       kPhaseBegin);
    if (st != SPINSIM_OK) return res->status = st;
    // the ordered product of the range: the top node of its chain tree
    const int n = req->spin_x2 + 1;
    double top[18];
    if (c.K > 0) {
        const Group& g = plan.groups[0];
        const ChainGeom cg = chain_geom(c.K);
        const char* src = static_cast<const char*>(h->arena.buf.p) + g.chain_off + g.chain.agg[cg.top];
        if (cudaMemcpyAsync(top, src, (size_t)op_doubles(req->spin_x2) * sizeof(double), cudaMemcpyDeviceToHost,
                            stream) != cudaSuccess)
            return res->status = SPINSIM_E_CUDA;
    }
    if (cudaStreamSynchronize(stream) != cudaSuccess) return res->status = SPINSIM_E_CUDA;
    if (c.K == 0) {
        for (int i = 0; i < 2 * n * n; i++) agg[i] = (i % (2 * n + 2) == 0) ? 1.0 : 0.0;
    } else if (n == 3) {
        for (int i = 0; i < 18; i++) agg[i] = top[i];
    } else {
        // SU(2) (alpha, beta) -> [[alpha, -conj(beta)], [beta, conj(alpha)]]
        const double ar = top[0], ai = top[1], br = top[2], bi = top[3];
        const double m[8] = {ar, ai, -br, bi, br, bi, ar, -ai};
        for (int i = 0; i < 8; i++) agg[i] = m[i];
    }
    h->range_req = *req;
    h->range_res = res;
    h->range_plan = plan;
    h->range_checked = checked;
    h->range_open = true;
    h->last.kernels_launched = kernels;
    res->n_samples = c.K;
    return SPINSIM_OK;
}

int spinsim_range_finish(spinsim_handle h, const double* psi_in, void* stream_v)
{
    if (!h || !psi_in || !h->range_open) return SPINSIM_E_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return SPINSIM_E_CUDA;
    h->range_open = false;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const int n = h->range_req.spin_x2 + 1;
    double nrm = 0.0;
    for (int i = 0; i < 2 * n; i++) {
        if (!std::isfinite(psi_in[i])) return SPINSIM_E_ARG;
        nrm += psi_in[i] * psi_in[i];
    }
    if (std::fabs(std::sqrt(nrm) - 1.0) > 1e-10) return SPINSIM_E_NORM;
    spinsim_request req = h->range_req;
    for (int i = 0; i < 6; i++) req.psi0[i] = i < 2 * n ? psi_in[i] : 0.0;
    h->last = spinsim_launch_info{};
    h->last.integrate_ms = -1.0;
    h->last.chain_ms = -1.0;
    h->prof_groups = 0;
    int kernels = 0;
    int st = run_batch(h, &req, h->range_res, h->range_checked, h->range_plan, stream, h->arena, h->pinned,
                       h->ev_pinned, false, &kernels, false, kPhaseFinish);
    h->last.kernels_launched = kernels;
    if (st != SPINSIM_OK) h->range_res->status = st;
    return st;
}

int spinsim_range_entering_state(int32_t spin_x2, const double* aggs, int32_t rank, const double* psi_init,
                                 double* psi_out)
{
    if ((spin_x2 != 1 && spin_x2 != 2) || rank < 0 || !psi_init || !psi_out || (rank > 0 && !aggs))
        return SPINSIM_E_ARG;
    const int n = spin_x2 + 1;
    double psi[6] = {}, nrm = 0.0;
    for (int i = 0; i < 2 * n; i++) {
        if (!std::isfinite(psi_init[i])) return SPINSIM_E_ARG;
        psi[i] = psi_init[i];
        nrm += psi[i] * psi[i];
    }
    if (std::fabs(std::sqrt(nrm) - 1.0) > 1e-10) return SPINSIM_E_NORM;
    // psi <- A_r psi for r = 0 .. rank - 1 (later ranges on the left), FP64,
    // renormalised after each range as every written state is
    for (int r = 0; r < rank; r++) {
        const double* A = aggs + (size_t)r * 2 * n * n;
        double out[6] = {};
        for (int i = 0; i < n; i++) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < n; j++) {
                const double ar = A[2 * (i * n + j)], ai = A[2 * (i * n + j) + 1];
                if (!std::isfinite(ar) || !std::isfinite(ai)) return SPINSIM_E_ARG;
                re += ar * psi[2 * j] - ai * psi[2 * j + 1];
                im += ar * psi[2 * j + 1] + ai * psi[2 * j];
            }
            out[2 * i] = re;
            out[2 * i + 1] = im;
        }
        double n2 = 0.0;
        for (int i = 0; i < 2 * n; i++) n2 += out[i] * out[i];
        if (!(n2 > 0.0)) return SPINSIM_E_ARG;
        const double inv = 1.0 / std::sqrt(n2);
        for (int i = 0; i < 2 * n; i++) psi[i] = out[i] * inv;
    }
    for (int i = 0; i < 2 * n; i++) psi_out[i] = psi[i];
    return SPINSIM_OK;
}

int spinsim_debug_bounds(int32_t device, uint64_t* word)
{
    if (!word) return SPINSIM_E_ARG;
    *word = 0;
#ifdef SPINSIM_BOUNDS
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(device) != cudaSuccess) return SPINSIM_E_CUDA;
    const uint64_t a = bounds_word_integrate(true), b = bounds_word_chain(true), c = bounds_word_static(true);
    if (prev >= 0) cudaSetDevice(prev);
    if (a == ~0ULL || b == ~0ULL || c == ~0ULL) return SPINSIM_E_CUDA;
    *word = a | b | c;
    return SPINSIM_OK;
#else
    (void)device;
    return SPINSIM_E_UNSUPPORTED;
#endif
}

int spinsim_last_launch(spinsim_handle h, spinsim_launch_info* info)
{
    if (!h || !info) return SPINSIM_E_ARG;
    if (h->prof_groups > 0) {
        double ti = 0.0, tc = 0.0;
        for (int g = 0; g < h->prof_groups; g++) {
            if (cudaEventSynchronize(h->prof[g][2]) != cudaSuccess) return SPINSIM_E_CUDA;
            float a = 0.f, b = 0.f;
            cudaEventElapsedTime(&a, h->prof[g][0], h->prof[g][1]);
            cudaEventElapsedTime(&b, h->prof[g][1], h->prof[g][2]);
            ti += a;
            tc += b;
        }
        h->last.integrate_ms = ti;
        h->last.chain_ms = tc;
    }
    *info = h->last;
    return SPINSIM_OK;
}

// ------------------------------------------------------------------ serving
// Continuous batching: requests wait in FIFO order until a stream slot is
// free and their scratch fits in the serving pool; every batch's scratch is a
// piece of that one pool.  The pool grows (cudaFree + cudaMalloc, which
// synchronise the device) only while no served batch is in flight, so no
// allocation ever stalls work already on the device, and the pool plus the
// main arena never exceed the handle's budget.
static constexpr size_t kPoolMinBytes = size_t(64) << 20;

static int serving_init(spinsim_s* h)
{
    if (!h->slots.empty()) return SPINSIM_OK;
    const int n_slots = 4;
    h->slots.resize(n_slots);
    for (Slot& s : h->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess)
            return SPINSIM_E_CUDA;
    }
    return SPINSIM_OK;
}

// First fit of `len` bytes (a multiple of 256) in the pool's free pieces.
static bool pool_carve(spinsim_s* h, size_t len, size_t* off)
{
    for (auto it = h->pool_free.begin(); it != h->pool_free.end(); ++it)
        if (it->second >= len) {
            const size_t o = it->first, rest = it->second - len;
            h->pool_free.erase(it);
            if (rest) h->pool_free[o + len] = rest;
            h->pool_in_use += len;
            *off = o;
            return true;
        }
    return false;
}

// Give a piece back, merging it with free neighbours.
static void pool_return(spinsim_s* h, size_t off, size_t len)
{
    if (!len) return;
    h->pool_in_use -= len;
    auto next = h->pool_free.lower_bound(off);
    if (next != h->pool_free.end() && off + len == next->first) {
        len += next->second;
        next = h->pool_free.erase(next);
    }
    if (next != h->pool_free.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second == off) {
            prev->second += len;
            return;
        }
    }
    h->pool_free[off] = len;
}

static size_t pool_largest_free(const spinsim_s* h)
{
    size_t m = 0;
    for (const auto& f : h->pool_free) m = std::max(m, f.second);
    return m;
}

// Replace the (idle) pool by one of at least `need` bytes: twice the old
// size or kPoolMinBytes when the budget allows.  The main arena is given
// back first when it leaves too little of the budget.
static int pool_grow(spinsim_s* h, size_t need)
{
    if (need > h->budget) return SPINSIM_E_NOMEM;
    int st = release_pool(h);
    if (st != SPINSIM_OK) return st;
    if (h->arena.buf.cap > h->budget - need) {
        drop_graph(h);   // the handle's graph refers to the arena
        h->range_open = false;
        st = release_device(h, h->arena.buf);
        if (st != SPINSIM_OK) return st;
    }
    const size_t room = h->budget - h->arena.buf.cap;
    size_t cap = round_up(std::max({need, 2 * h->pool.cap, kPoolMinBytes}), size_t(1) << 20);
    cap = std::min(cap, room);
    if (cap < need) return SPINSIM_E_NOMEM;
    if (inject_alloc_failure(h) || cudaMalloc(&h->pool.p, cap) != cudaSuccess) {
        cudaGetLastError();
        h->pool.p = nullptr;
        return SPINSIM_E_NOMEM;
    }
    h->pool.cap = cap;
    note_held(h);
    h->pool_free[0] = cap;
    return SPINSIM_OK;
}

static void ticket_done(spinsim_s* h, int64_t id, Ticket& tk)
{
    tk.state = 2;
    h->done_order.push_back(id);
}

// Retire finished batches, then launch pending requests on free slots while
// their scratch fits in the pool (FIFO: the head waits until it fits).
static int serving_pump(spinsim_s* h)
{
    for (Slot& s : h->slots) {
        if (!s.busy) continue;
        cudaError_t q = cudaEventQuery(s.done);
        if (q == cudaErrorNotReady) continue;
        const int st = q == cudaSuccess ? SPINSIM_OK : SPINSIM_E_CUDA;
        if (q != cudaSuccess) cudaGetLastError();
        for (int64_t t : s.tickets) {
            auto it = h->tickets.find(t);
            if (it == h->tickets.end()) continue;
            if (st != SPINSIM_OK) it->second.res->status = st;
            ticket_done(h, t, it->second);
        }
        h->requests_in_flight -= (int64_t)s.tickets.size();
        s.tickets.clear();
        pool_return(h, s.off, s.len);
        s.off = s.len = 0;
        s.busy = false;
    }
    for (Slot& s : h->slots) {
        if (h->pending.empty()) break;
        if (s.busy) continue;
        size_t room = pool_largest_free(h);
        {
            Ticket& head = h->tickets[h->pending.front()];
            if (head.bytes > room && !serving_busy(h)) {
                // nothing in flight: the pool may be replaced without stalling work
                const int st = pool_grow(h, head.bytes);
                if (st != SPINSIM_OK) {
                    head.res->status = st;
                    ticket_done(h, h->pending.front(), head);
                    h->pending.pop_front();
                    continue;
                }
                room = pool_largest_free(h);
            }
        }
        std::vector<spinsim_request> reqs;
        std::vector<spinsim_result> res;
        std::vector<int64_t> ids;
        std::vector<Checked> checked;
        Footprint fp(h->cfg.precision);
        while (!h->pending.empty()) {
            const int64_t t = h->pending.front();
            Ticket& tk = h->tickets[t];
            Checked c = check_request(&tk.req);
            if (c.status == SPINSIM_OK) c.status = precision_status(h->cfg, tk.req);
            if (c.status == SPINSIM_OK) c.variant = request_variant(h->cfg, tk.req, c.K, c.L);
            Footprint next = fp;
            next.add(tk.req.spin_x2, c.variant, c.K, tk.req.field.n_tones, tk.staged);
            if (next.total() > room) break;
            fp = next;
            h->pending.pop_front();
            reqs.push_back(tk.req);
            res.push_back(*tk.res);
            ids.push_back(t);
            checked.push_back(c);
        }
        if (ids.empty()) break;   // the head waits for a batch to retire
        Plan plan;
        build_plan(reqs.data(), res.data(), (int64_t)reqs.size(), checked, h->cfg.precision, false, plan, h->cfg.direct_host_outputs != 0);
        size_t off = 0;
        int st = SPINSIM_OK;
        if (!pool_carve(h, round_up(plan.total, 256), &off)) st = SPINSIM_E_NOMEM;   // total() bounds plan.total
        int kernels = 0;
        if (st == SPINSIM_OK) {
            s.off = off;
            s.len = round_up(plan.total, 256);
            Arena piece;
            piece.buf.p = static_cast<char*>(h->pool.p) + off;
            piece.buf.cap = s.len;
            st = run_batch(h, reqs.data(), res.data(), checked, plan, s.stream, piece, s.pinned, s.done, false,
                           &kernels);
        }
        for (size_t q = 0; q < ids.size(); q++) {
            Ticket& tk = h->tickets[ids[q]];
            tk.state = 1;
            tk.res->trotter_squares = res[q].trotter_squares;
            if (st != SPINSIM_OK) tk.res->status = st;
        }
        if (cudaEventRecord(s.done, s.stream) != cudaSuccess) return SPINSIM_E_CUDA;
        s.tickets = ids;
        s.busy = true;
        h->requests_in_flight += (int64_t)ids.size();
    }
    return SPINSIM_OK;
}

int spinsim_submit(spinsim_handle h, const spinsim_request* req, spinsim_result* res, int64_t* ticket)
{
    if (!h || !req || !res || !ticket) return SPINSIM_E_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return SPINSIM_E_CUDA;
    h->range_open = false;
    int st = serving_init(h);
    if (st != SPINSIM_OK) return st;
    Checked c = check_request(req);
    if (c.status == SPINSIM_OK) c.status = precision_status(h->cfg, *req);
    if (c.status == SPINSIM_OK) {
        if (!res->states) c.status = SPINSIM_E_ARG;
        else if (res->capacity < c.K) c.status = SPINSIM_E_CAPACITY;
    }
    if (c.status == SPINSIM_OK) c.flags |= precision_flags(h->cfg.precision, h->cfg.rotating_frame, *req);
    res->status = c.status;
    res->flags = c.flags;
    res->trotter_squares = 0;
    res->n_samples = c.status == SPINSIM_OK ? c.K : 0;
    const int64_t id = h->next_ticket++;
    Ticket tk;
    tk.req = *req;
    tk.res = res;
    tk.slot = -1;
    tk.state = 0;
    tk.staged = 0;
    tk.bytes = 0;
    if (c.status == SPINSIM_OK) {
        tk.staged = staging_bytes(*req, *res, c.K, false, h->cfg.direct_host_outputs != 0);
        Footprint fp(h->cfg.precision);
        fp.add(req->spin_x2, request_variant(h->cfg, *req, c.K, c.L), c.K, req->field.n_tones, tk.staged);
        tk.bytes = round_up(fp.total(), 256);
        if (tk.bytes > h->budget) c.status = res->status = SPINSIM_E_NOMEM;   // could never be admitted
    }
    h->tickets[id] = tk;
    *ticket = id;
    if (c.status != SPINSIM_OK) {
        ticket_done(h, id, h->tickets[id]);
        return c.status;
    }
    h->pending.push_back(id);
    return serving_pump(h);
}

int spinsim_poll(spinsim_handle h, int64_t ticket, int32_t wait_us)
{
    if (!h) return SPINSIM_E_ARG;
    if (cudaSetDevice(h->device) != cudaSuccess) return SPINSIM_E_CUDA;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        int st = serving_pump(h);
        if (st != SPINSIM_OK) return st;
        auto it = h->tickets.find(ticket);
        if (it == h->tickets.end()) return SPINSIM_E_ARG;
        if (it->second.state == 2) {
            h->tickets.erase(it);
            return SPINSIM_OK;
        }
        if (wait_us <= 0) return SPINSIM_PENDING;
        auto dt = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        if (dt >= wait_us) return SPINSIM_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int spinsim_poll_any(spinsim_handle h, int64_t* tickets, int64_t capacity, int32_t wait_us, int64_t* n_done)
{
    if (!h || !n_done || capacity < 0 || (capacity > 0 && !tickets)) return SPINSIM_E_ARG;
    *n_done = 0;
    if (cudaSetDevice(h->device) != cudaSuccess) return SPINSIM_E_CUDA;
    auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        int st = serving_pump(h);
        if (st != SPINSIM_OK) return st;
        while (*n_done < capacity && !h->done_order.empty()) {
            const int64_t t = h->done_order.front();
            h->done_order.pop_front();
            auto it = h->tickets.find(t);
            if (it == h->tickets.end()) continue;   // already reported by spinsim_poll
            h->tickets.erase(it);
            tickets[(*n_done)++] = t;
        }
        if (*n_done > 0 || capacity == 0) return SPINSIM_OK;
        if (wait_us <= 0) return SPINSIM_PENDING;
        auto dt = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
        if (dt >= wait_us) return SPINSIM_E_TIMEOUT;
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

int spinsim_memory(spinsim_handle h, spinsim_memory_info* info)
{
    if (!h || !info) return SPINSIM_E_ARG;
    info->budget = (int64_t)h->budget;
    info->held = (int64_t)h->held;
    info->peak_held = (int64_t)h->peak_held;
    info->arena = (int64_t)h->arena.buf.cap;
    info->pool = (int64_t)h->pool.cap;
    info->pool_in_use = (int64_t)h->pool_in_use;
    info->pending = (int64_t)h->pending.size();
    info->in_flight = h->requests_in_flight;
    return SPINSIM_OK;
}

}  // extern "C"
