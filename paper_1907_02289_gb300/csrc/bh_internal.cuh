// bh_internal.cuh -- context layout and helpers shared by the libbh.so
// translation units (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/bh.h"

namespace bh {

constexpr int kLevels = 21;                    // key depth: 21 octal digits, 63 bits
constexpr uint32_t kQMax = (1u << kLevels) - 1;

// Device status word bits (set by kernels, read at synchronising calls).
constexpr int kStatNonFinite = 1;
constexpr int kStatListOverflow = 2;
constexpr int kStatTimeout = 4;
constexpr int kStatBounds = 8;  // an internal index check failed (access skipped)
constexpr int kStatRange = 16;  // a contact term outside the fixed-point accumulator's range
constexpr int kStatAxis = 32;   // cylindrical key frame with a particle on the axis (r = 0)

// Sizes of a device-sized list build (a list-constructing step captured as
// one graph: nothing is read back while it runs), in Ctx::d_sz.
constexpr int kSzLvl = 0;                   // kLevels + 3 words: first node of each level, then the node count
constexpr int kSzNg = kLevels + 3;          // group count
constexpr int kSzOvf = kSzNg + 1;           // overflow bits
constexpr int kSzNeedNodes = kSzOvf + 1;    // nodes wanted when the node capacity ran out (a lower bound)
constexpr int kSzWords = 32;
constexpr unsigned long long kOvfNodes = 1, kOvfLists = 2;

// Device buffer that only grows.
template <typename T>
struct DBuf {
    T* p = nullptr;
    size_t cap = 0;
};

struct Ctx;
int fail(Ctx* c, int code, const char* fmt, ...);

// cudaMalloc-backed growth; returns BH_OK or BH_E_NOMEM (with message).
int grow_raw(Ctx* c, void** p, size_t* cap, size_t bytes_needed, const char* what, bool keep);
template <typename T>
int grow(Ctx* c, DBuf<T>& b, size_t n, const char* what, bool keep = false) {
    size_t cap_bytes = b.cap * sizeof(T);
    int rc = grow_raw(c, (void**)&b.p, &cap_bytes, n * sizeof(T), what, keep);
    b.cap = cap_bytes / sizeof(T);
    return rc;
}

// Per-node packed record read by the walk (one 32-byte load per visit):
// a = (qlo.x | level << 21 | leaf flag, qlo.y | leaf count << 21, qlo.z,
// successor of the subtree or -1), b = (qhi.xyz, first child, or for a leaf
// its first particle).  A leaf count of kWalkCntMax means "that many or
// more": the walk then reads the node's end.
struct WalkNode {
    uint4 a, b;
};
constexpr uint32_t kWalkLeaf = 1u << 26;
constexpr uint32_t kWalkCntMax = (1u << 11) - 1;

// Launch tuning of the FP32 force kernel (bh_set_tuning / the autotuner).
struct Tuning {
    int chunk = 96;          // largest i-chunk per warp pass: 32, 64 or 96 particles
    int warps = 4;           // warps per block, 1..8
    int sched = BH_SCHED_DYNAMIC;
    int order_by_cost = 1;   // within a size class, largest estimated cost first
    int graph = 0;           // capture list-reusing steps of bh_step in a CUDA graph
    int order_window = 0;    // > 0: size-class order within windows of this many groups
    int graph_contact_room = 0;  // > 0: contact candidates a graph step may hold (0: automatic)
    int graph_room = 25;         // percent of room over the last build in a list-constructing graph step
};

struct Ctx {
    bh_params prm;
    Tuning tune;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    std::string err;

    // state
    int64_t n = 0;
    bool have_tree = false, have_lists = false, have_acc = false;
    int64_t k_eval = 0;        // force evaluations done (drives the rebuild schedule)
    int64_t evals_since_build = 0, n_rebuilds = 0;
    int64_t n_launches = 0;    // kernels launched by this context

    // optional CUDA-event timing of the force kernel (one event pair per launch)
    // and of every stage (BH_STAGE_*)
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_force;
    struct StageEv {
        int stage;
        cudaEvent_t a, b;
    };
    std::vector<StageEv> ev_stage;       // recorded, not yet read
    std::vector<int> stage_open;         // indices into ev_stage of stages begun, not ended
    double stage_ms[BH_N_STAGES] = {};   // read stage times, summed since the last reset
    int64_t stage_calls[BH_N_STAGES] = {};

    // list capacity (bh_params.list_capacity; 0 = none) and the sizes a build
    // that exceeded it needed
    bool list_overflowed = false;
    int64_t need_pp = 0, need_pc = 0, need_jj = 0;

    // patches: independent particle sets, each with its own root box and
    // tree (a forest whose roots are nodes 0..n_patches-1); 1 for one set
    int n_patches = 1;
    std::vector<int64_t> h_off;         // particle offsets of the patches (n_patches + 1)
    DBuf<int64_t> d_off;                // the same on the device
    DBuf<uint32_t> tile_meta;           // sort tiles per patch (4 words per tile), n_patches > 1
    int64_t n_tiles = 0;
    DBuf<uint2> box_map;                // root-box blocks of the patches: (patch, block within it)
    DBuf<int> box_poff;                 // first root-box block of each patch (n_patches + 1)
    int n_box_blocks = 0;
    DBuf<long long> d_rcq;              // per patch walk contact threshold
    DBuf<long long> d_rfar;             // per patch far threshold of the split expansion
    DBuf<long long> d_period;           // per patch phi period in grid cells (cylindrical frame; 0 = none)

    // status and small device scalars
    int* d_status = nullptr;
    double* d_box = nullptr;   // per patch: lo[3], L, S, spare x3 (8 doubles)
    unsigned long long* d_small = nullptr;  // scan totals etc. (64 words)

    // keys and sort
    DBuf<uint64_t> key[2];
    DBuf<uint32_t> idx[2];
    int key_cur = 0;           // buffer holding the sorted keys / perm
    DBuf<uint32_t> sort_hist;
    DBuf<uint32_t> digit_hist; // 8 x 256 global digit counts
    DBuf<double> pscratch;     // permutation scratch (8 arrays x 8 bytes per particle)
    DBuf<double> cyl;          // cylindrical frame: phi[n], r[n]
    DBuf<unsigned long long> box_part;  // root-box partials (6 per block, as ordered integers)
    DBuf<uint8_t> scan_tmp;

    // tree
    int64_t n_nodes = 0;
    std::vector<int64_t> lvl_start;  // node id range of each level (size depth+2)
    DBuf<uint8_t> level, nchild;
    DBuf<uint32_t> begin, end;
    DBuf<int32_t> parent, first_child;
    DBuf<uint32_t> qlo, qhi;         // 3 per node
    DBuf<WalkNode> wnode;
    DBuf<uint32_t> split_cnt;        // per node of a level
    DBuf<uint32_t> split_off;
    DBuf<uint32_t> split_bnd;        // 9 per node of a level

    // moments
    DBuf<double> M, cx, cy, cz, Q;   // Q: 6 per node
    DBuf<float4> cell32;             // 3 per node: (c_hi, M), (c_lo, Qxx), (Qxy, Qxz, Qyy, Qyz)
    DBuf<float> cell32lo;            // per node: exact mass - M of the record (FP32)
    DBuf<float4> phi, plo;           // per particle FP32 split: (x_hi, m), (x_lo, 0)
    DBuf<uint2> refine;                 // (particle, list slot) queued for the refinement pass
    DBuf<float> cbnd;                   // particles with contact candidates: FP32 bound,
    DBuf<uint32_t> cslot;               // list slot,
    DBuf<unsigned> cflag;               // and a flag the post-contact check claims
    DBuf<unsigned long long> contacts;  // (i, j) contact candidates for the FP64 pass
    DBuf<double> diag;                   // diagnostic partial sums
    DBuf<double> pot;                    // per-particle potential when the caller passes none
    DBuf<unsigned long long> contact_acc;  // per particle fixed-point contact sums (3 per particle)
    int64_t n_contacts = 0;
    int64_t n_refined = 0;              // particles the refinement pass re-evaluated (last read)
    bool refine_pending = false;        // an evaluation ran since n_refined was read
    bool contact_stats = false;         // the device contact counters hold an FP32 evaluation's counts

    // groups
    int64_t n_groups = 0;
    DBuf<int32_t> gmark;             // per particle: group node starting here, or -1
    DBuf<uint32_t> gflag, gpos;
    DBuf<int32_t> groups;            // node ids ordered by begin
    DBuf<int32_t> order;             // force-kernel processing order of groups
    DBuf<unsigned long long> order_cnt;  // order buckets: counts/starts and cursors
    DBuf<uint64_t> ord_key[2];           // windowed order: sort keys
    DBuf<uint32_t> ord_idx[2];
    DBuf<uint32_t> ord_scratch;
    int sort_attr_device = -1;           // device the sort kernel's smem limit was raised on
    int f32_attr_device = -1;            // device the FP32 kernels' smem limit was raised on
    unsigned f32_blocks = 0;             // grid of the last FP32 force launch
    DBuf<unsigned long long> warp_time;  // per warp (start, end) of the last persistent launch
    int64_t warp_time_n = 0;
    bool capturing = false;              // issuing work into a stream capture
    cudaGraphExec_t graph_exec = nullptr;  // the captured list-reusing step
    cudaStream_t cap_stream = nullptr;   // private stream the step is captured on
    // host-buffer stepping: positions, masses and ids are final once the last
    // evaluation's tree/moments stage is enqueued; their copy back is
    // enqueued right there, on a second stream, so that it overlaps the force
    // kernel (the host waits after that kernel to size the contact pass)
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t pos_event = nullptr;
    bool want_pos_event = false, pos_event_recorded = false;
    bool early_now = false;              // the evaluation being run is the call's last
    const bh_particles* early_dst = nullptr;  // host arrays of the early copy
    const bh_particles* early_src = nullptr;  // device arrays it copies from
    bool early_ids = true;               // the early copy includes masses and ids
    int64_t h2d_bytes = 0, d2h_bytes = 0;  // copied by bh_step_host so far
    bool graph_ok = false;               // graph_exec matches the current lists and arrays
    bh_particles graph_p{};              // particle arrays the graph was captured with
    int64_t graph_launches = 0;          // kernels in the graph

    // device-sized list builds: a list-constructing step of bh_step issued as
    // one graph (graph tuning on), its buffers sized from the previous build
    unsigned long long* d_sz = nullptr;  // kSzWords device words (level bounds, group count, overflow)
    bool dev_build = false;              // issuing a device-sized build (no size read-backs)
    const unsigned long long* abort = nullptr;  // while issuing the forces and kick of such a step: its
                                                // overflow bits (nonzero: those kernels do nothing)
    int64_t cap_nodes = 0;               // node capacity of the build being issued
    int64_t dev_slots = 0;               // groups with a list slot in it
    cudaGraphExec_t rgraph_exec = nullptr;  // the captured list-constructing step
    bool rgraph_ok = false;              // rgraph_exec matches the arrays and capacities
    bh_particles rgraph_p{};
    int64_t rgraph_launches = 0;
    int64_t rgraph_cap[5] = {};          // nodes, slots, P, C, JJ it was captured with
    int64_t rgraph_walk_cap[2] = {};     // and list slot sizes
    cudaStream_t body_stream[2] = {nullptr, nullptr};  // its conditional bodies are captured on these
    // force-kernel timing inside step graphs: event-record nodes around the
    // kernel, given fresh events before each launch while timing is on
    struct GraphTiming {
        cudaGraph_t g = nullptr;             // the graph the executable was instantiated from
        cudaGraphNode_t node[2] = {nullptr, nullptr};
        bool have = false;
    };
    GraphTiming gt_reuse, gt_rebuild, gt_tmp;
    GraphTiming* gt_cur = nullptr;           // the graph being captured
    cudaEvent_t gt_idle[2] = {nullptr, nullptr};  // recorded by those nodes while timing is off
    int64_t n_graph_builds = 0;          // list builds that ran inside a graph
    int64_t n_graph_build_redos = 0;     // of those, builds redone eagerly after a capacity ran out
    int64_t n_graph_captures = 0;        // step graphs captured

    // lists
    int64_t n_pp = 0, n_pc = 0, n_jj = 0;
    int64_t n_int_pp = 0, n_int_pc = 0;
    int64_t n_int_pp_far = 0;            // FP32 path: pp interactions with far list particles
    DBuf<int64_t> cnt_p, cnt_c, cnt_j;   // per group counts, then offsets (ng + 1)
    DBuf<int64_t> cnt_jm;                // FP32 path: per group index of the first far list particle
    DBuf<int32_t> stash_p, stash_c;      // per group list slots of the one-walk build
    int64_t walk_cap_p = 0, walk_cap_c = 0;  // their sizes (0: count and fill walks)
    int64_t n_one_walk_builds = 0;       // list builds whose lists came from one walk
    DBuf<int32_t> P, C;
    DBuf<uint32_t> JJ;
    DBuf<int64_t> ipp;                   // per group interaction counts (scratch)

    // host-buffer stepping
    DBuf<double> hbuf;                   // 10 arrays of n doubles
    DBuf<int64_t> hid;
};

// ---- CUDA error plumbing -------------------------------------------------
#define BH_CUDA(c, call)                                                              \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return ::bh::fail((c), BH_E_CUDA, "%s failed: %s (%s:%d)", #call,          \
                              cudaGetErrorString(e_), __FILE__, __LINE__);            \
    } while (0)
#define BH_TRY(expr)                 \
    do {                             \
        int r_ = (expr);             \
        if (r_ != BH_OK) return r_;  \
    } while (0)
#define BH_LAUNCH(c)                                                                  \
    do {                                                                              \
        cudaError_t e_ = cudaGetLastError();                                          \
        if (e_ != cudaSuccess)                                                        \
            return ::bh::fail((c), BH_E_CUDA, "kernel launch failed: %s (%s:%d)",      \
                              cudaGetErrorString(e_), __FILE__, __LINE__);            \
        (c)->n_launches++;                                                            \
    } while (0)

inline unsigned blocks_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    return (unsigned)(b < 1 ? 1 : b);
}

// ---- stage entry points (one translation unit each) ------------------------
// scan.cu: exclusive prefix sums; *total written to d_total (device) if given.
// With dn, the element count is read on the device (*dn, at most n).
int scan_u32(Ctx* c, const uint32_t* in, uint32_t* out, int64_t n, unsigned long long* d_total,
             const unsigned long long* dn = nullptr);
int scan_i64(Ctx* c, const int64_t* in, int64_t* out, int64_t n, unsigned long long* d_total,
             const unsigned long long* dn = nullptr);
int64_t scan_sums_count(int64_t n);
cudaError_t scan_u32_with(cudaStream_t s, const uint32_t* in, uint32_t* out, int64_t n, uint32_t* sums);

// sort.cu
int stage_keys(Ctx* c, const bh_particles* p);     // root box + keys (+ status on NaN)
int stage_sort(Ctx* c);                            // stable LSD radix sort of (key, idx)
int stage_permute(Ctx* c, bh_particles* p);        // gather particle arrays into key order
int setup_patches(Ctx* c, int n_patches, const int64_t* off);  // bh_api.cu
int64_t sort_tiles_for(const std::vector<int64_t>& off, std::vector<uint32_t>* meta);  // sort.cu
// context-free sort over caller buffers (sort.cu); scratch >= sort_scratch_words(n) words
int64_t sort_scratch_words(int64_t n);
cudaError_t sort_setup_device();
cudaError_t sort_pairs_with(cudaStream_t s, uint64_t* keys, uint32_t* idx, uint64_t* ktmp, uint32_t* itmp,
                            int64_t n, uint32_t* scratch);

// tree.cu
int stage_octree(Ctx* c);                          // level-by-level split; sets n_nodes
int stage_octree_dev(Ctx* c);                      // the same, device-sized (c->dev_build)
int stage_boxes(Ctx* c);                           // integer boxes + walk records
int stage_moments(Ctx* c, const bh_particles* p);  // M, c, Q (+ FP32 cell records)
int stage_moments64(Ctx* c, const bh_particles* p);  // FP64 M, c, Q whatever the precision
int stage_groups(Ctx* c);                          // groups ordered by begin

// walk.cu
int stage_lists(Ctx* c);                           // walk (count, fill) + particle expansion
int stage_lists_dev_walk(Ctx* c);                  // device-sized: walk, offsets, room check
int stage_lists_dev_fill(Ctx* c);                  // device-sized: lists, expansion, group order

// force.cu
int stage_split(Ctx* c, const bh_particles* p);    // FP32 hi/lo split of particles
int build_order32(Ctx* c);                         // FP32 kernel's group order (per list build)
int stage_force(Ctx* c, bh_particles* p, bool add_central);
int stage_potential(Ctx* c, const bh_particles* p, double* phi, double* W);  // self-gravity potential (FP64)

// bh_api.cu: force-kernel and stage timing (no-ops unless enabled, or while
// capturing a graph); stage_end closes the innermost stage begun
int timing_begin(Ctx* c);
int timing_end(Ctx* c);
int stage_begin(Ctx* c, int stage);
int stage_end(Ctx* c);

// update.cu
int stage_kick(Ctx* c, bh_particles* p, double h);
int stage_kick_drift(Ctx* c, bh_particles* p, double h, double dt);
int stage_diagnostics(Ctx* c, const bh_particles* p, double* host_out);  // 11 sums to the host

}  // namespace bh
