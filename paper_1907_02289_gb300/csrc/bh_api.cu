// bh_api.cu -- the C ABI of libbh.so (declared in include/bh.h): context
// life cycle, the list-constructing / list-reusing schedule of Sec. 4.2,
// the leapfrog driver and the read-back functions.
#include <stdarg.h>

#include <algorithm>
#include <cmath>

#include "bh_internal.cuh"

namespace bh {

int fail(Ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

int grow_raw(Ctx* c, void** p, size_t* cap, size_t need, const char* what, bool keep) {
    if (need <= *cap && *p) return BH_OK;
    // a captured step cannot allocate: its buffers are sized before capture
    if (c->capturing) return fail(c, BH_E_STATE, "%s would have to grow inside a captured step", what);
    void* q = nullptr;
    // A buffer that has to grow again (list sizes vary a little from one
    // build to the next) gets a quarter of headroom: each regrowth costs a
    // stream synchronisation, an allocation and a free in the middle of a step.
    size_t bytes = *p ? need + need / 4 : need;
    if (bytes < 256) bytes = 256;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, BH_E_NOMEM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what,
                    cudaGetErrorString(e));
    }
    if (*p) {
        if (keep && *cap) {
            e = cudaMemcpyAsync(q, *p, *cap, cudaMemcpyDeviceToDevice, c->stream);
            if (e != cudaSuccess) return fail(c, BH_E_CUDA, "copy while growing %s: %s", what, cudaGetErrorString(e));
        }
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return fail(c, BH_E_CUDA, "sync while growing %s: %s", what, cudaGetErrorString(e));
        cudaFree(*p);
    }
    *p = q;
    *cap = bytes;
    return BH_OK;
}

static cudaEvent_t take_event(Ctx* c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

// While a step graph is captured: an event-record node (recording a
// placeholder event) before (k = 0) or after (k = 1) the force kernel, whose
// event each launch then sets (launch_graph).
static int graph_timing_node(Ctx* c, int k) {
    Ctx::GraphTiming* gt = c->gt_cur;
    if (!gt || !c->gt_idle[k]) return BH_OK;
    BH_CUDA(c, cudaEventRecordWithFlags(c->gt_idle[k], c->stream, cudaEventRecordExternal));
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    BH_CUDA(c, cudaStreamGetCaptureInfo(c->stream, &st, nullptr, nullptr, &deps, nullptr, &nd));
    if (nd != 1) return fail(c, BH_E_STATE, "timing node of a captured step: %zu dependencies", nd);
    gt->node[k] = deps[0];
    gt->have = k == 1 && gt->node[0] != nullptr;
    return BH_OK;
}

int timing_begin(Ctx* c) {
    if (c->capturing) return graph_timing_node(c, 0);
    if (!c->timing) return BH_OK;
    cudaEvent_t a = take_event(c), b = take_event(c);
    if (!a || !b) return fail(c, BH_E_CUDA, "cudaEventCreate failed");
    BH_CUDA(c, cudaEventRecord(a, c->stream));
    c->ev_force.push_back({a, b});
    return BH_OK;
}

int timing_end(Ctx* c) {
    if (c->capturing) return graph_timing_node(c, 1);
    if (!c->timing || c->ev_force.empty()) return BH_OK;
    BH_CUDA(c, cudaEventRecord(c->ev_force.back().second, c->stream));
    return BH_OK;
}

int stage_begin(Ctx* c, int stage) {
    if (!c->timing || c->capturing) return BH_OK;
    cudaEvent_t a = take_event(c), b = take_event(c);
    if (!a || !b) return fail(c, BH_E_CUDA, "cudaEventCreate failed");
    BH_CUDA(c, cudaEventRecord(a, c->stream));
    c->stage_open.push_back((int)c->ev_stage.size());
    c->ev_stage.push_back({stage, a, b});
    return BH_OK;
}

int stage_end(Ctx* c) {
    if (!c->timing || c->capturing || c->stage_open.empty()) return BH_OK;
    const int k = c->stage_open.back();
    c->stage_open.pop_back();
    BH_CUDA(c, cudaEventRecord(c->ev_stage[k].b, c->stream));
    return BH_OK;
}

// Read the recorded stage events into the sums: all of them after
// synchronising the stream (wait), or, without waiting, those already
// complete (in recording order).
static int read_stage_events(Ctx* c, bool wait) {
    if (c->ev_stage.empty()) return BH_OK;
    if (wait) BH_CUDA(c, cudaStreamSynchronize(c->stream));
    size_t keep = c->stage_open.empty() ? c->ev_stage.size() : (size_t)c->stage_open.front();
    if (!wait)
        for (size_t k = 0; k < keep; ++k) {
            const cudaError_t q = cudaEventQuery(c->ev_stage[k].b);
            if (q == cudaErrorNotReady) {
                keep = k;
                break;
            }
            BH_CUDA(c, q);
        }
    for (size_t k = 0; k < keep; ++k) {
        float ms = 0.f;
        BH_CUDA(c, cudaEventElapsedTime(&ms, c->ev_stage[k].a, c->ev_stage[k].b));
        c->stage_ms[c->ev_stage[k].stage] += ms;
        c->stage_calls[c->ev_stage[k].stage]++;
        c->ev_pool.push_back(c->ev_stage[k].a);
        c->ev_pool.push_back(c->ev_stage[k].b);
    }
    c->ev_stage.erase(c->ev_stage.begin(), c->ev_stage.begin() + keep);
    for (int& k : c->stage_open) k -= (int)keep;
    return BH_OK;
}

// Run a stage under its timing events.
#define BH_STAGE(c, id, expr)              \
    do {                                   \
        BH_TRY(stage_begin((c), (id)));    \
        BH_TRY(expr);                      \
        BH_TRY(stage_end(c));              \
    } while (0)

// Patch layout: offsets on host and device, per-patch root boxes, sort tiles.
int setup_patches(Ctx* c, int n_patches, const int64_t* off) {
    c->n_patches = n_patches;
    c->h_off.assign(off, off + n_patches + 1);
    BH_TRY(grow(c, c->d_off, (size_t)n_patches + 1, "patch offsets"));
    BH_CUDA(c, cudaMemcpyAsync(c->d_off.p, c->h_off.data(), c->h_off.size() * sizeof(int64_t),
                               cudaMemcpyHostToDevice, c->stream));
    std::vector<uint32_t> meta;
    std::vector<uint2> map;
    std::vector<int> poff;
    if (n_patches > 1) {
        c->n_tiles = sort_tiles_for(c->h_off, &meta);
        BH_TRY(grow(c, c->tile_meta, meta.size(), "sort tile table"));
        BH_CUDA(c, cudaMemcpyAsync(c->tile_meta.p, meta.data(), meta.size() * sizeof(uint32_t),
                                   cudaMemcpyHostToDevice, c->stream));
        // root-box blocks in proportion to the patch sizes (at least one
        // each; about four per SM in all)
        const double total = (double)(off[n_patches] - off[0]);
        const double want = 4.0 * c->num_sms;
        poff.push_back(0);
        for (int q = 0; q < n_patches; ++q) {
            const int64_t sz = off[q + 1] - off[q];
            const int nbq = (int)std::max<double>(1.0, std::ceil(want * (double)sz / total));
            for (int j = 0; j < nbq; ++j) map.push_back(make_uint2((unsigned)q, (unsigned)j));
            poff.push_back((int)map.size());
        }
        c->n_box_blocks = (int)map.size();
        BH_TRY(grow(c, c->box_map, map.size(), "root-box block map"));
        BH_TRY(grow(c, c->box_poff, poff.size(), "root-box block offsets"));
        BH_CUDA(c, cudaMemcpyAsync(c->box_map.p, map.data(), map.size() * sizeof(uint2), cudaMemcpyHostToDevice,
                                   c->stream));
        BH_CUDA(c, cudaMemcpyAsync(c->box_poff.p, poff.data(), poff.size() * sizeof(int), cudaMemcpyHostToDevice,
                                   c->stream));
    }
    BH_CUDA(c, cudaStreamSynchronize(c->stream));  // (the host tables above outlive no call)
    return BH_OK;
}

namespace {

template <typename T>
void release(DBuf<T>& b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
}

int check_params(Ctx* c, const bh_params* p) {
    if (!p) return fail(c, BH_E_INVAL, "params is NULL");
    if (!(p->theta >= 0.0) || !std::isfinite(p->theta)) return fail(c, BH_E_INVAL, "theta must be >= 0");
    if (p->n_g < 1) return fail(c, BH_E_INVAL, "n_g must be >= 1");
    if (p->n_leaf < 1 || p->n_leaf > p->n_g) return fail(c, BH_E_INVAL, "need 1 <= n_leaf <= n_g");
    if (p->order != 1 && p->order != 2) return fail(c, BH_E_INVAL, "order must be 1 or 2");
    if (p->precision != BH_PREC_FP64 && p->precision != BH_PREC_FP32)
        return fail(c, BH_E_INVAL, "precision must be BH_PREC_FP64 or BH_PREC_FP32");
    if (p->rebuild_every < 1) return fail(c, BH_E_INVAL, "rebuild_every must be >= 1");
    if (p->key_frame != 0 && p->key_frame != 1)
        return fail(c, BH_E_INVAL, "key_frame must be 0 (Cartesian) or 1 (cylindrical)");
    if (!(p->eps >= 0.0) || !(p->r_coll >= 0.0) || !(p->dt >= 0.0))
        return fail(c, BH_E_INVAL, "eps, r_coll and dt must be >= 0");
    if (p->list_capacity < 0) return fail(c, BH_E_INVAL, "list_capacity must be >= 0");
    if (!std::isfinite(p->omega)) return fail(c, BH_E_INVAL, "omega must be finite");
    return BH_OK;
}

int check_particles(Ctx* c, const bh_particles* p, bool need_v) {
    if (!p) return fail(c, BH_E_INVAL, "particles is NULL");
    if (p->n < 1 || p->n >= ((int64_t)1 << 31)) return fail(c, BH_E_INVAL, "need 1 <= n < 2^31 (n = %lld)", (long long)p->n);
    if (!p->x || !p->y || !p->z || !p->m || !p->ax || !p->ay || !p->az)
        return fail(c, BH_E_INVAL, "x, y, z, m, ax, ay, az must be set");
    if (need_v && (!p->vx || !p->vy || !p->vz)) return fail(c, BH_E_INVAL, "vx, vy, vz must be set");
    return BH_OK;
}

int read_status(Ctx* c) {
    int st = 0;
    BH_CUDA(c, cudaMemcpyAsync(&st, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st) BH_CUDA(c, cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream));
    if (st & kStatNonFinite) return fail(c, BH_E_INVAL, "non-finite particle coordinate");
    if (st & kStatAxis) return fail(c, BH_E_INVAL, "the cylindrical key frame needs every particle off the axis (r > 0)");
    if (st & kStatListOverflow) return fail(c, BH_E_LIST_OVERFLOW, "list buffer overflow");
    if (st & kStatTimeout) return fail(c, BH_E_TIMEOUT, "device wait timed out");
    if (st & kStatBounds) return fail(c, BH_E_STATE, "internal index check failed (access skipped)");
    if (st & kStatRange)
        return fail(c, BH_E_INVAL, "a contact acceleration term reached 1024 or was not finite (kappa, eta too large?)");
    return BH_OK;
}

int build_tree(Ctx* c, bh_particles* p) {
    BH_TRY(check_particles(c, p, true));
    if (c->n_patches > 1 && p->n != c->h_off.back())
        return fail(c, BH_E_INVAL, "n = %lld but the patches hold %lld particles", (long long)p->n,
                    (long long)c->h_off.back());
    c->n = p->n;
    c->have_tree = c->have_lists = false;
    if (c->n_patches == 1 && (c->h_off.size() != 2 || c->h_off[1] != p->n)) {
        const int64_t off[2] = {0, p->n};
        BH_TRY(setup_patches(c, 1, off));
    }
    BH_STAGE(c, BH_STAGE_KEYS, stage_keys(c, p));
    BH_TRY(read_status(c));  // non-finite coordinates; a particle on the axis of the cylindrical frame
    BH_STAGE(c, BH_STAGE_SORT, stage_sort(c));
    BH_STAGE(c, BH_STAGE_PERMUTE, stage_permute(c, p));
    BH_TRY(stage_begin(c, BH_STAGE_TREE));
    BH_TRY(stage_octree(c));
    BH_TRY(stage_boxes(c));
    BH_TRY(stage_end(c));
    BH_TRY(stage_moments(c, p));
    BH_STAGE(c, BH_STAGE_GROUPS, stage_groups(c));
    c->have_tree = true;
    return BH_OK;
}

int make_lists(Ctx* c) {
    if (!c->have_tree) return fail(c, BH_E_STATE, "bh_make_lists needs a tree (call bh_build_tree)");
    BH_STAGE(c, BH_STAGE_LISTS, stage_lists(c));
    c->have_lists = true;
    c->graph_ok = false;
    c->evals_since_build = 0;
    c->n_rebuilds++;
    return BH_OK;
}

// One force evaluation of the stepping schedule: list-constructing when
// k_eval % rebuild_every == 0, list-reusing otherwise.
int evaluate(Ctx* c, bh_particles* p) {
    if (c->k_eval % c->prm.rebuild_every == 0 || !c->have_lists) {
        BH_TRY(build_tree(c, p));
        BH_TRY(make_lists(c));
    } else {
        BH_TRY(stage_moments(c, p));
    }
    if (c->want_pos_event && c->early_now) {  // x..id are final for this step from here on
        BH_CUDA(c, cudaEventRecord(c->pos_event, c->stream));
        c->pos_event_recorded = true;
        if (c->early_dst) {  // copy them back while the force kernel runs
            const bh_particles& h = *c->early_dst;
            const bh_particles& d = *c->early_src;
            const size_t nb = (size_t)d.n * sizeof(double);
            BH_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->pos_event, 0));
            BH_CUDA(c, cudaMemcpyAsync(h.x, d.x, nb, cudaMemcpyDeviceToHost, c->copy_stream));
            BH_CUDA(c, cudaMemcpyAsync(h.y, d.y, nb, cudaMemcpyDeviceToHost, c->copy_stream));
            BH_CUDA(c, cudaMemcpyAsync(h.z, d.z, nb, cudaMemcpyDeviceToHost, c->copy_stream));
            if (c->early_ids) {  // masses and ids change only when the evaluations reorder
                BH_CUDA(c, cudaMemcpyAsync(h.m, d.m, nb, cudaMemcpyDeviceToHost, c->copy_stream));
                BH_CUDA(c, cudaMemcpyAsync(h.id, d.id, (size_t)d.n * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                           c->copy_stream));
            }
        }
    }
    BH_TRY(stage_force(c, p, true));
    c->k_eval++;
    c->evals_since_build++;
    return BH_OK;
}

// Step-graph timing: the placeholder events (made before any capture), the
// launch that sets the force kernel's timing events, and the graph kept for
// its node handles.
int ensure_graph_events(Ctx* c) {
    for (cudaEvent_t& e : c->gt_idle)
        if (!e) BH_CUDA(c, cudaEventCreate(&e));
    return BH_OK;
}

int launch_graph(Ctx* c, cudaGraphExec_t exec, const Ctx::GraphTiming& gt) {
    if (gt.have) {
        cudaEvent_t a = c->gt_idle[0], b = c->gt_idle[1];
        const bool timed = c->timing;
        if (timed) {
            a = take_event(c);
            b = take_event(c);
            if (!a || !b) return fail(c, BH_E_CUDA, "cudaEventCreate failed");
        }
        BH_CUDA(c, cudaGraphExecEventRecordNodeSetEvent(exec, gt.node[0], a));
        BH_CUDA(c, cudaGraphExecEventRecordNodeSetEvent(exec, gt.node[1], b));
        BH_CUDA(c, cudaGraphLaunch(exec, c->stream));
        if (timed) c->ev_force.push_back({a, b});
        return BH_OK;
    }
    BH_CUDA(c, cudaGraphLaunch(exec, c->stream));
    return BH_OK;
}

void keep_graph(Ctx::GraphTiming& dst, Ctx::GraphTiming& src) {
    if (dst.g && dst.g != src.g) cudaGraphDestroy(dst.g);
    dst = src;
    src = Ctx::GraphTiming{};
}

bool same_arrays(const bh_particles& a, const bh_particles& b) {
    return a.x == b.x && a.y == b.y && a.z == b.z && a.vx == b.vx && a.vy == b.vy && a.vz == b.vz && a.m == b.m &&
           a.id == b.id && a.ax == b.ax && a.ay == b.ay && a.az == b.az && a.n == b.n;
}

// One list-reusing step (kick-drift, moment refresh, forces, kick) as a CUDA
// graph launch; the graph is captured on the first such step after a list
// build (or when the arrays change) and updated in place when possible.
int graph_reuse_step(Ctx* c, bh_particles* p) {
    const double dt = c->prm.dt;
    if (!c->graph_ok || !same_arrays(c->graph_p, *p)) {
        // inside the graph the contact pass cannot grow its buffer: leave room
        // for twice the candidates of the last eager evaluation
        if (c->prm.precision == BH_PREC_FP32 && c->prm.r_coll > 0.0) {
            const size_t want = c->tune.graph_contact_room > 0 ? (size_t)c->tune.graph_contact_room
                                                               : (size_t)(2 * c->n_contacts + 65536);
            if (c->contacts.cap < want) BH_TRY(grow(c, c->contacts, want, "contact pairs"));
        }
        // capture on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the context's stream
        if (!c->cap_stream) BH_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        BH_TRY(ensure_graph_events(c));
        c->gt_tmp = Ctx::GraphTiming{};
        c->gt_cur = &c->gt_tmp;
        cudaGraph_t g = nullptr;
        const cudaStream_t s0 = c->stream;
        c->stream = c->cap_stream;
        {
            const cudaError_t eb = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
            if (eb != cudaSuccess) {
                c->stream = s0;
                BH_CUDA(c, eb);
            }
        }
        c->capturing = true;
        const int64_t l0 = c->n_launches;
        int rc = stage_kick_drift(c, p, 0.5 * dt, dt);
        if (rc == BH_OK) rc = stage_moments(c, p);
        if (rc == BH_OK) rc = stage_force(c, p, true);
        if (rc == BH_OK) rc = stage_kick(c, p, 0.5 * dt);
        c->capturing = false;
        c->gt_cur = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
        c->stream = s0;
        c->graph_launches = c->n_launches - l0;
        c->n_launches = l0;
        if (rc != BH_OK) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (ec != cudaSuccess) return fail(c, BH_E_CUDA, "stream capture of the step failed: %s", cudaGetErrorString(ec));
        // an update keeps the executable's nodes (those of the graph it was
        // instantiated from, kept for the timing nodes)
        bool updated = false;
        if (c->graph_exec) {
            cudaGraphExecUpdateResultInfo info;
            updated = cudaGraphExecUpdate(c->graph_exec, g, &info) == cudaSuccess;
            if (!updated) {
                cudaGetLastError();
                cudaGraphExecDestroy(c->graph_exec);
                c->graph_exec = nullptr;
            }
        }
        cudaError_t ei = cudaSuccess;
        if (updated) {
            cudaGraphDestroy(g);
        } else {
            ei = cudaGraphInstantiate(&c->graph_exec, g, 0);
            c->gt_tmp.g = g;
            keep_graph(c->gt_reuse, c->gt_tmp);
        }
        if (ei != cudaSuccess) {
            c->graph_exec = nullptr;
            return fail(c, BH_E_CUDA, "cudaGraphInstantiate failed: %s", cudaGetErrorString(ei));
        }
        c->graph_ok = true;
        c->graph_p = *p;
        ++c->n_graph_captures;
    }
    BH_TRY(launch_graph(c, c->graph_exec, c->gt_reuse));
    c->n_launches += c->graph_launches;
    c->refine_pending = c->prm.precision == BH_PREC_FP32;  // its count is read when asked for
    c->k_eval++;
    c->evals_since_build++;
    return BH_OK;
}

// ---- list-constructing steps as one graph ---------------------------------
// With graph tuning 1, a list-constructing step of bh_step (kick-drift, keys,
// sort, permutation, tree, moments, groups, walk, lists, forces, contact and
// refinement passes, kick) is one graph launch.  Its buffers are sized before
// capture from the previous build, with room to grow; the step reads nothing
// back while it runs (sizes stay on the device, kSz*).  Two conditional nodes
// guard the build: the work after the tree runs only if the nodes fitted
// their capacity, the list writing after the walk only if the lists fitted
// theirs.  The forces and the final kick sit at the graph's top level (where
// the force kernel's timing nodes can be) and do nothing when an overflow bit
// is set.  A step that outgrew its buffers thus stops with positions kicked
// and drifted and particles reordered; the host, which reads the sizes at the
// step's end, grows the buffers and finishes it eagerly, with the same result.

__global__ void k_cond_set(cudaGraphConditionalHandle h, const unsigned long long* sz, unsigned long long mask) {
    if (threadIdx.x == 0) cudaGraphSetConditional(h, (sz[kSzOvf] & mask) ? 0u : 1u);
}

namespace {

// The graph being captured on c->stream and its current dependencies.
int capture_state(Ctx* c, cudaGraph_t* g, const cudaGraphNode_t** deps, size_t* nd) {
    cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
    BH_CUDA(c, cudaStreamGetCaptureInfo(c->stream, &st, nullptr, g, deps, nullptr, nd));
    if (st != cudaStreamCaptureStatusActive) return fail(c, BH_E_STATE, "stream capture is not active");
    return BH_OK;
}

// Set h from the device (non-zero when none of the mask's overflow bits is
// set), then add an IF node on h to the graph being captured on c->stream and
// issue work into its body, captured on body_stream.
template <class F>
int capture_if(Ctx* c, unsigned long long mask, cudaStream_t body_stream, F issue) {
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    BH_TRY(capture_state(c, &g, &deps, &nd));
    cudaGraphConditionalHandle h;
    BH_CUDA(c, cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    k_cond_set<<<1, 32, 0, c->stream>>>(h, c->d_sz, mask);
    BH_LAUNCH(c);
    BH_TRY(capture_state(c, &g, &deps, &nd));
    cudaGraphNodeParams prm = {};
    prm.type = cudaGraphNodeTypeConditional;
    prm.conditional.handle = h;
    prm.conditional.type = cudaGraphCondTypeIf;
    prm.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    BH_CUDA(c, cudaGraphAddNode(&node, g, deps, nullptr, nd, &prm));
    BH_CUDA(c, cudaStreamUpdateCaptureDependencies(c->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = prm.conditional.phGraph_out[0];
    BH_CUDA(c, cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    const cudaStream_t s0 = c->stream;
    c->stream = body_stream;
    const int rc = issue();
    c->stream = s0;
    cudaGraph_t out = nullptr;
    const cudaError_t e = cudaStreamEndCapture(body_stream, &out);
    BH_TRY(rc);
    BH_CUDA(c, e);
    return BH_OK;
}

struct HostSizes {
    int64_t n_nodes, n_groups;
    int key_cur;
    std::vector<int64_t> lvl_start;
};

// Buffers of a device-sized build, grown before capture (nothing can grow
// inside it): node arrays to the node capacity, group arrays to one group
// per particle, slots, lists and the FP32 pass buffers.
int size_dev_build(Ctx* c, const int64_t cap[5]) {
    const int64_t n = c->n, nodes = cap[0];
    const bool f32 = c->prm.precision == BH_PREC_FP32;
    for (auto* b : {&c->level, &c->nchild}) BH_TRY(grow(c, *b, (size_t)nodes, "node arrays"));
    for (auto* b : {&c->begin, &c->end}) BH_TRY(grow(c, *b, (size_t)nodes, "node arrays"));
    for (auto* b : {&c->parent, &c->first_child}) BH_TRY(grow(c, *b, (size_t)nodes, "node arrays"));
    BH_TRY(grow(c, c->qlo, 3 * (size_t)nodes, "node qlo"));
    BH_TRY(grow(c, c->qhi, 3 * (size_t)nodes, "node qhi"));
    BH_TRY(grow(c, c->wnode, (size_t)nodes, "walk records"));
    BH_TRY(grow(c, c->split_cnt, (size_t)nodes, "split counts"));
    BH_TRY(grow(c, c->split_bnd, 9 * (size_t)nodes, "split bounds"));
    BH_TRY(grow(c, c->split_off, (size_t)nodes / 256 + 2, "split tile sums"));
    if (f32) {
        BH_TRY(grow(c, c->cell32, 3 * (size_t)nodes, "FP32 cell records"));
        BH_TRY(grow(c, c->cell32lo, (size_t)nodes, "FP32 cell mass corrections"));
    } else {
        for (auto* b : {&c->M, &c->cx, &c->cy, &c->cz}) BH_TRY(grow(c, *b, (size_t)nodes, "moments"));
        BH_TRY(grow(c, c->Q, 6 * (size_t)nodes, "moments Q"));
    }
    BH_TRY(grow(c, c->groups, (size_t)n + 1, "groups"));
    for (auto* b : {&c->cnt_p, &c->cnt_c, &c->cnt_j, &c->cnt_jm})
        BH_TRY(grow(c, *b, (size_t)n + 1, "list offsets"));
    BH_TRY(grow(c, c->order, (size_t)n + 1, "group order"));
    // scans over up to n group counts (8-byte words, 2048 per tile)
    BH_TRY(grow(c, c->scan_tmp, ((size_t)n / 2048 + 2) * sizeof(int64_t), "scan block sums"));
    BH_TRY(grow(c, c->stash_p, (size_t)std::max<int64_t>(1, cap[1] * c->walk_cap_p), "stashed particle lists"));
    BH_TRY(grow(c, c->stash_c, (size_t)std::max<int64_t>(1, cap[1] * c->walk_cap_c), "stashed cell lists"));
    BH_TRY(grow(c, c->P, (size_t)cap[2] + 1, "particle lists"));
    BH_TRY(grow(c, c->C, (size_t)cap[3] + 1, "cell lists"));
    BH_TRY(grow(c, c->JJ, (size_t)cap[4] + 1, "list particle indices"));
    if (f32 && c->prm.r_coll > 0.0) {
        const size_t want = c->tune.graph_contact_room > 0 ? (size_t)c->tune.graph_contact_room
                                                           : (size_t)(2 * c->n_contacts + 65536);
        if (c->contacts.cap < want) BH_TRY(grow(c, c->contacts, want, "contact pairs"));
    }
    return BH_OK;
}

int capture_rebuild(Ctx* c, bh_particles* p) {
    const double dt = c->prm.dt;
    // capacities: the last build's sizes with graph_room percent to grow
    const int64_t r = c->tune.graph_room;
    auto room = [r](int64_t v) { return v + v * r / 100 + 64; };
    int64_t cap[5];
    cap[0] = room(c->n_nodes);
    cap[1] = std::min<int64_t>(c->n, room(c->n_groups));
    cap[2] = room(c->n_pp);
    cap[3] = room(c->n_pc);
    cap[4] = room(c->n_jj);
    BH_TRY(size_dev_build(c, cap));
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaStream_t* ss[3] = {&c->cap_stream, &c->body_stream[0], &c->body_stream[1]};
    for (cudaStream_t* q : ss)
        if (!*q) BH_CUDA(c, cudaStreamCreateWithFlags(q, cudaStreamNonBlocking));
    BH_TRY(ensure_graph_events(c));
    const HostSizes keep{c->n_nodes, c->n_groups, c->key_cur, c->lvl_start};
    c->cap_nodes = cap[0];
    c->gt_tmp = Ctx::GraphTiming{};
    c->gt_cur = &c->gt_tmp;
    c->dev_slots = cap[1];
    const cudaStream_t s0 = c->stream;
    c->stream = c->cap_stream;
    {  // (relaxed: the conditional nodes' handles are made while capturing)
        const cudaError_t eb = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed);
        if (eb != cudaSuccess) {
            c->stream = s0;
            BH_CUDA(c, eb);
        }
    }
    c->capturing = true;
    c->dev_build = true;
    const int64_t l0 = c->n_launches;
    int rc = stage_kick_drift(c, p, 0.5 * dt, dt);
    if (rc == BH_OK) rc = stage_keys(c, p);
    if (rc == BH_OK) rc = stage_sort(c);
    if (rc == BH_OK) rc = stage_permute(c, p);
    if (rc == BH_OK) rc = stage_octree(c);
    if (rc == BH_OK)
        rc = capture_if(c, kOvfNodes, c->body_stream[0], [&]() -> int {
            BH_TRY(stage_boxes(c));
            BH_TRY(stage_moments(c, p));
            BH_TRY(stage_groups(c));
            BH_TRY(stage_lists_dev_walk(c));
            return capture_if(c, kOvfLists, c->body_stream[1], [&]() -> int { return stage_lists_dev_fill(c); });
        });
    // forces and kick at the top level (where the force kernel's timing
    // nodes may sit): they read the overflow bits and do nothing when the
    // build outgrew its buffers; the contact and refinement passes then find
    // no candidates
    c->abort = c->d_sz + kSzOvf;
    if (rc == BH_OK) rc = stage_force(c, p, true);
    if (rc == BH_OK) rc = stage_kick(c, p, 0.5 * dt);
    c->abort = nullptr;
    c->capturing = false;
    c->dev_build = false;
    c->gt_cur = nullptr;
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(c->stream, &g);
    c->stream = s0;
    c->rgraph_launches = c->n_launches - l0;
    c->n_launches = l0;
    c->n_nodes = keep.n_nodes;
    c->n_groups = keep.n_groups;
    c->lvl_start = keep.lvl_start;
    if (rc != BH_OK || ec != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        c->key_cur = keep.key_cur;  // nothing ran: the sorted keys are where they were
        if (rc != BH_OK) return rc;
        return fail(c, BH_E_CUDA, "stream capture of the list-constructing step failed: %s", cudaGetErrorString(ec));
    }
    if (c->rgraph_exec) {
        cudaGraphExecDestroy(c->rgraph_exec);
        c->rgraph_exec = nullptr;
    }
    const cudaError_t ei = cudaGraphInstantiate(&c->rgraph_exec, g, 0);
    c->gt_tmp.g = g;  // kept with the executable (its timing nodes)
    keep_graph(c->gt_rebuild, c->gt_tmp);
    if (ei != cudaSuccess) {
        c->rgraph_exec = nullptr;
        cudaGetLastError();
        return fail(c, BH_E_CUDA, "cudaGraphInstantiate of the list-constructing step failed: %s",
                    cudaGetErrorString(ei));
    }
    ++c->n_graph_captures;
    for (int k = 0; k < 5; ++k) c->rgraph_cap[k] = cap[k];
    c->rgraph_walk_cap[0] = c->walk_cap_p;
    c->rgraph_walk_cap[1] = c->walk_cap_c;
    c->rgraph_ok = true;
    c->rgraph_p = *p;
    return BH_OK;
}

// The captured step still leaves the last build at least half its room (and
// slot sizes within a tenth), on the same arrays.
bool rebuild_graph_fits(const Ctx* c, const bh_particles* p) {
    if (!c->rgraph_ok || !c->rgraph_exec || !same_arrays(c->rgraph_p, *p)) return false;
    const int64_t now[5] = {c->n_nodes, c->n_groups, c->n_pp, c->n_pc, c->n_jj};
    for (int k = 0; k < 5; ++k)
        if (now[k] + now[k] * c->tune.graph_room / 200 > c->rgraph_cap[k]) return false;
    return c->walk_cap_p <= c->rgraph_walk_cap[0] + c->rgraph_walk_cap[0] / 10 &&
           c->walk_cap_c <= c->rgraph_walk_cap[1] + c->rgraph_walk_cap[1] / 10;
}

}  // namespace

int graph_rebuild_step(Ctx* c, bh_particles* p) {
    if (!rebuild_graph_fits(c, p)) BH_TRY(capture_rebuild(c, p));
    BH_TRY(launch_graph(c, c->rgraph_exec, c->gt_rebuild));
    c->n_launches += c->rgraph_launches;
    unsigned long long sz[kSzWords], sm[24];
    BH_CUDA(c, cudaMemcpyAsync(sz, c->d_sz, sizeof(sz), cudaMemcpyDeviceToHost, c->stream));
    BH_CUDA(c, cudaMemcpyAsync(sm, c->d_small, sizeof(sm), cudaMemcpyDeviceToHost, c->stream));
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    BH_TRY(read_status(c));
    ++c->n_graph_builds;
    if (sz[kSzOvf] != 0) {
        // a capacity ran out: the step stopped after the kick-drift and the
        // reordering; grow at the next capture and finish it eagerly
        ++c->n_graph_build_redos;
        c->rgraph_ok = false;  // captured again from the eager build's sizes
        c->have_tree = c->have_lists = false;
        BH_TRY(evaluate(c, p));
        return stage_kick(c, p, 0.5 * c->prm.dt);
    }
    // the sizes of the build, as an eager build leaves them
    c->n_nodes = (int64_t)sz[kSzLvl + kLevels + 2];
    c->lvl_start.assign(1, 0);
    for (int l = 0; l <= kLevels && sz[kSzLvl + l + 1] > sz[kSzLvl + l]; ++l)
        c->lvl_start.push_back((int64_t)sz[kSzLvl + l + 1]);
    c->n_groups = (int64_t)sz[kSzNg];
    c->n_pp = (int64_t)sm[0];
    c->n_pc = (int64_t)sm[1];
    c->n_jj = (int64_t)sm[2];
    c->n_int_pp = (int64_t)sm[8];
    c->n_int_pc = (int64_t)sm[9];
    c->n_int_pp_far = c->prm.precision == BH_PREC_FP32 ? (int64_t)sm[10] : 0;
    if (sm[11] == 0) ++c->n_one_walk_builds;
    c->walk_cap_p = (int64_t)(((sm[12] + sm[12] / 4 + 4) + 3) & ~3ull);
    c->walk_cap_c = (int64_t)(((sm[13] + sm[13] / 4 + 4) + 3) & ~3ull);
    if (c->prm.precision == BH_PREC_FP32 && c->prm.r_coll > 0.0) c->n_contacts = (int64_t)sm[16];
    c->have_tree = c->have_lists = true;
    c->list_overflowed = false;
    c->graph_ok = false;  // the list-reusing graph follows the new lists
    c->n_rebuilds++;
    c->evals_since_build = 1;
    c->k_eval++;
    c->refine_pending = c->prm.precision == BH_PREC_FP32;
    return BH_OK;
}

int check_tuning(Ctx* c, const bh_tuning* t) {
    if (!t) return fail(c, BH_E_INVAL, "tuning is NULL");
    if (t->n_g < c->prm.n_leaf) return fail(c, BH_E_INVAL, "n_g must be >= n_leaf");
    if (t->chunk != 32 && t->chunk != 64 && t->chunk != 96) return fail(c, BH_E_INVAL, "chunk must be 32, 64 or 96");
    if (t->warps < 1 || t->warps > 8) return fail(c, BH_E_INVAL, "warps must be 1..8");
    if (t->sched < BH_SCHED_GRID || t->sched > BH_SCHED_DYNAMIC) return fail(c, BH_E_INVAL, "unknown schedule");
    if ((t->order_by_cost != 0 && t->order_by_cost != 1) || t->graph < 0 || t->graph > 2)
        return fail(c, BH_E_INVAL, "order_by_cost must be 0 or 1, graph 0, 1 or 2");
    if (t->order_window < 0) return fail(c, BH_E_INVAL, "order_window must be >= 0");
    if (t->graph_contact_room < 0) return fail(c, BH_E_INVAL, "graph_contact_room must be >= 0");
    if (t->graph_room < 0 || t->graph_room > 1000) return fail(c, BH_E_INVAL, "graph_room must be 0..1000");
    return BH_OK;
}

void apply_tuning(Ctx* c, const bh_tuning* t) {
    const bool relist = t->n_g != c->prm.n_g || t->chunk != c->tune.chunk || t->order_by_cost != c->tune.order_by_cost;
    if (t->n_g != c->prm.n_g) c->have_lists = false;
    c->prm.n_g = t->n_g;
    c->tune.chunk = t->chunk;
    c->tune.warps = t->warps;
    c->tune.sched = t->sched;
    c->tune.order_by_cost = t->order_by_cost;
    c->tune.graph = t->graph;
    c->tune.order_window = t->order_window;
    c->tune.graph_contact_room = t->graph_contact_room;
    c->tune.graph_room = t->graph_room;
    c->graph_ok = false;
    c->rgraph_ok = false;
    (void)relist;
}

void read_tuning(const Ctx* c, bh_tuning* t) {
    t->n_g = c->prm.n_g;
    t->chunk = c->tune.chunk;
    t->warps = c->tune.warps;
    t->sched = c->tune.sched;
    t->order_by_cost = c->tune.order_by_cost;
    t->graph = c->tune.graph;
    t->order_window = c->tune.order_window;
    t->graph_contact_room = c->tune.graph_contact_room;
    t->graph_room = c->tune.graph_room;
}

// Elapsed device time of fn() on the context's stream (ms).
template <class F>
int time_ms(Ctx* c, F fn, double* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    BH_CUDA(c, cudaEventCreate(&a));
    cudaError_t e = cudaEventCreate(&b);
    if (e != cudaSuccess) {
        cudaEventDestroy(a);
        BH_CUDA(c, e);
    }
    int rc = BH_OK;
    e = cudaEventRecord(a, c->stream);
    if (e == cudaSuccess) rc = fn();
    if (e == cudaSuccess && rc == BH_OK) e = cudaEventRecord(b, c->stream);
    if (e == cudaSuccess && rc == BH_OK) e = cudaEventSynchronize(b);
    float f = 0.f;
    if (e == cudaSuccess && rc == BH_OK) e = cudaEventElapsedTime(&f, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (rc != BH_OK) return rc;
    BH_CUDA(c, e);
    *ms = f;
    return BH_OK;
}

int autotune(Ctx* c, bh_particles* p, double* best_ms) {
    BH_TRY(check_particles(c, p, true));
    const bool timing = c->timing;
    c->timing = false;
    bh_tuning cur;
    read_tuning(c, &cur);
    const int graph = cur.graph;
    cur.graph = 0;
    apply_tuning(c, &cur);
    double tb = 0.0;
    auto build = [&]() -> int {
        BH_TRY(build_tree(c, p));
        return make_lists(c);
    };
    auto force = [&]() -> int {
        BH_TRY(stage_moments(c, p));
        return stage_force(c, p, false);
    };
    // (1) launch settings on the current n_g, by force-evaluation time, one
    // knob at a time: schedule, warps per block, i-chunk, order window
    BH_TRY(time_ms(c, build, &tb));
    double best_f = 1e300;
    bh_tuning best = cur;
    // the first force evaluations after a list build run slower (fresh lists
    // and particle order), so each phase starts with untimed evaluations and
    // every candidate keeps the best of three
    auto settle = [&]() -> int {
        for (int w = 0; w < 2; ++w) BH_TRY(force());
        return BH_OK;
    };
    auto try_force = [&](const bh_tuning& t) -> int {
        const bool reorder = t.chunk != c->tune.chunk || t.order_window != c->tune.order_window;
        apply_tuning(c, &t);
        if (reorder && c->prm.precision == BH_PREC_FP32) BH_TRY(build_order32(c));
        double ms = 1e300;
        for (int rep = 0; rep < 3; ++rep) {
            double m = 0.0;
            BH_TRY(time_ms(c, force, &m));
            if (m < ms) ms = m;
        }
        if (ms < best_f) {
            best_f = ms;
            best = t;
        }
        return BH_OK;
    };
    BH_TRY(settle());
    if (c->prm.precision == BH_PREC_FP32) {
        for (int sc = BH_SCHED_GRID; sc <= BH_SCHED_DYNAMIC; ++sc) {
            bh_tuning t = best;
            t.sched = sc;
            BH_TRY(try_force(t));
        }
        const int warps[3] = {2, 4, 8}, chunks[3] = {32, 64, 96}, windows[3] = {0, 2048, 8192};
        for (int q = 0; q < 3; ++q) {
            bh_tuning t = best;
            t.warps = warps[q];
            BH_TRY(try_force(t));
        }
        for (int q = 0; q < 3; ++q) {
            bh_tuning t = best;
            t.chunk = chunks[q];
            BH_TRY(try_force(t));
        }
        for (int q = 0; q < 3; ++q) {
            bh_tuning t = best;
            t.order_window = windows[q];
            BH_TRY(try_force(t));
        }
    } else {
        BH_TRY(try_force(best));  // the FP64 kernel has no launch settings
    }
    // (2) n_g by the cost of a step: force time + list-build time / rebuild_every
    {
        double best_step = 1e300;
        bh_tuning best_ng = best;
        const int cand[5] = {64, 96, 128, 192, 256};
        for (int q = 0; q < 5; ++q) {
            if (cand[q] < c->prm.n_leaf) continue;
            bh_tuning t = best;
            t.n_g = cand[q];
            apply_tuning(c, &t);
            double b = 0.0, f = 1e300;
            BH_TRY(time_ms(c, build, &b));
            BH_TRY(settle());
            for (int rep = 0; rep < 3; ++rep) {
                double m = 0.0;
                BH_TRY(time_ms(c, force, &m));
                if (m < f) f = m;
            }
            const double step = f + b / c->prm.rebuild_every;
            if (step < best_step) {
                best_step = step;
                best_ng = t;
            }
        }
        best = best_ng;
        if (best_ms) *best_ms = best_step;
    }
    // (3) the i-chunk and the order window together, on the chosen n_g (the
    // best chunk depends on the group sizes -- groups of 2 x 96 run uniform
    // chunks -- and on the window)
    if (c->prm.precision == BH_PREC_FP32) {
        apply_tuning(c, &best);
        double b = 0.0;
        BH_TRY(time_ms(c, build, &b));
        BH_TRY(settle());
        best_f = 1e300;
        BH_TRY(try_force(best));
        const double f_best = best_f;
        const int chunks[3] = {32, 64, 96}, windows[3] = {0, 2048, 8192};
        const bh_tuning base = best;
        for (int q = 0; q < 3; ++q)  // all pairs: the best chunk depends on the window
            for (int w = 0; w < 3; ++w) {
                bh_tuning t = base;
                t.chunk = chunks[q];
                t.order_window = windows[w];
                BH_TRY(try_force(t));
            }
        if (best_ms) *best_ms += best_f - f_best;
    }
    best.graph = graph;
    apply_tuning(c, &best);
    BH_TRY(build_tree(c, p));
    BH_TRY(make_lists(c));
    BH_TRY(stage_force(c, p, true));
    c->k_eval = 1;
    c->evals_since_build = 1;
    c->have_acc = true;
    c->timing = timing;
    return read_status(c);
}

}  // namespace
}  // namespace bh

using bh::Ctx;

extern "C" {

static int create_ctx(const char* who, const bh_params* p, int n_patches, const int64_t* offsets, void* stream,
                      bh_ctx** out) {
    if (!out) return BH_E_INVAL;
    *out = nullptr;
    Ctx tmp;
    int rc = bh::check_params(&tmp, p);
    if (rc == BH_OK && n_patches > 1) {
        if (!offsets) {
            rc = bh::fail(&tmp, BH_E_INVAL, "offsets is NULL");
        } else if (offsets[0] != 0) {
            rc = bh::fail(&tmp, BH_E_INVAL, "offsets[0] must be 0");
        } else {
            for (int q = 0; q < n_patches && rc == BH_OK; ++q)
                if (offsets[q + 1] <= offsets[q])
                    rc = bh::fail(&tmp, BH_E_INVAL, "patch %d is empty or offsets decrease", q);
            if (rc == BH_OK && offsets[n_patches] >= ((int64_t)1 << 31))
                rc = bh::fail(&tmp, BH_E_INVAL, "total particle count must be < 2^31");
        }
    }
    if (rc != BH_OK) {
        fprintf(stderr, "%s: %s\n", who, tmp.err.c_str());
        return rc;
    }
    Ctx* c = new Ctx();
    c->prm = *p;
    c->stream = (cudaStream_t)stream;
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_box, 8 * sizeof(double) * (size_t)n_patches);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_small, 64 * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&c->d_sz, bh::kSzWords * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_sz, 0, bh::kSzWords * sizeof(unsigned long long), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_status, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        fprintf(stderr, "%s: CUDA error: %s\n", who, cudaGetErrorString(e));
        cudaGetLastError();
        bh_destroy((bh_ctx*)c);
        return BH_E_CUDA;
    }
    if (n_patches > 1 && (rc = bh::setup_patches(c, n_patches, offsets)) != BH_OK) {
        fprintf(stderr, "%s: %s\n", who, c->err.c_str());
        bh_destroy((bh_ctx*)c);
        return rc;
    }
    *out = (bh_ctx*)c;
    return BH_OK;
}

int bh_create(const bh_params* p, void* stream, bh_ctx** out) {
    return create_ctx("bh_create", p, 1, nullptr, stream, out);
}

int bh_batch_create(const bh_params* p, int n_patches, const int64_t* offsets, void* stream, bh_ctx** out) {
    if (n_patches < 1 || n_patches > 65535) {
        fprintf(stderr, "bh_batch_create: n_patches must be in 1..65535\n");
        if (out) *out = nullptr;
        return BH_E_INVAL;
    }
    if (n_patches == 1) return create_ctx("bh_batch_create", p, 1, nullptr, stream, out);
    return create_ctx("bh_batch_create", p, n_patches, offsets, stream, out);
}

int bh_destroy(bh_ctx* ctx) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_OK;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->rgraph_exec) cudaGraphExecDestroy(c->rgraph_exec);
    for (Ctx::GraphTiming* gt : {&c->gt_reuse, &c->gt_rebuild, &c->gt_tmp})
        if (gt->g) cudaGraphDestroy(gt->g);
    for (cudaEvent_t e : c->gt_idle)
        if (e) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaStream_t q : c->body_stream)
        if (q) cudaStreamDestroy(q);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->pos_event) cudaEventDestroy(c->pos_event);
    cudaFree(c->d_status);
    cudaFree(c->d_box);
    cudaFree(c->d_small);
    cudaFree(c->d_sz);
    using bh::release;
    release(c->d_off); release(c->tile_meta); release(c->box_map); release(c->box_poff); release(c->d_rcq); release(c->d_rfar); release(c->d_period); release(c->cyl); release(c->box_part); release(c->order_cnt); release(c->warp_time); release(c->contact_acc); release(c->diag); release(c->pot);
    for (int b = 0; b < 2; ++b) {
        release(c->ord_key[b]);
        release(c->ord_idx[b]);
    }
    release(c->ord_scratch);
    for (int b = 0; b < 2; ++b) {
        release(c->key[b]);
        release(c->idx[b]);
    }
    release(c->sort_hist); release(c->digit_hist); release(c->pscratch); release(c->scan_tmp);
    release(c->level); release(c->nchild); release(c->begin); release(c->end); release(c->parent);
    release(c->first_child); release(c->qlo); release(c->qhi); release(c->wnode); release(c->split_cnt);
    release(c->split_off); release(c->split_bnd); release(c->M); release(c->cx); release(c->cy);
    release(c->cz); release(c->Q); release(c->cell32); release(c->cell32lo); release(c->refine); release(c->cbnd); release(c->cslot); release(c->cflag); release(c->phi); release(c->plo); release(c->contacts); release(c->gmark);
    release(c->gflag); release(c->gpos); release(c->groups); release(c->order); release(c->cnt_p);
    release(c->cnt_c); release(c->cnt_j); release(c->cnt_jm); release(c->stash_p); release(c->stash_c); release(c->P); release(c->C); release(c->JJ); release(c->ipp);
    release(c->hbuf); release(c->hid);
    for (auto& pr : c->ev_force) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    delete c;
    return BH_OK;
}

const char* bh_last_error(const bh_ctx* ctx) {
    const Ctx* c = (const Ctx*)ctx;
    return c ? c->err.c_str() : "no context";
}

int bh_set_stream(bh_ctx* ctx, void* stream) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    c->stream = (cudaStream_t)stream;
    return BH_OK;
}

int bh_build_tree(bh_ctx* ctx, bh_particles* p) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    return bh::build_tree(c, p);
}

int bh_make_lists(bh_ctx* ctx) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    return bh::make_lists(c);
}

int bh_compute_forces(bh_ctx* ctx, bh_particles* p, int flags) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_lists) return bh::fail(c, BH_E_STATE, "bh_compute_forces needs lists (call bh_make_lists)");
    BH_TRY(bh::check_particles(c, p, true));
    if (p->n != c->n) return bh::fail(c, BH_E_INVAL, "particle count changed since the tree was built");
    BH_TRY(bh::stage_moments(c, p));
    BH_TRY(bh::stage_force(c, p, !(flags & BH_FORCE_TREE_ONLY)));
    c->evals_since_build++;
    return BH_OK;
}

int bh_step(bh_ctx* ctx, bh_particles* p, int nsteps) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (nsteps < 0) return bh::fail(c, BH_E_INVAL, "nsteps must be >= 0");
    BH_TRY(bh::check_particles(c, p, true));
    if (c->have_tree && p->n != c->n) return bh::fail(c, BH_E_INVAL, "particle count changed");
    const double dt = c->prm.dt;
    c->early_now = false;  // the initial evaluation is never the step's last
    if (!c->have_acc) {
        BH_TRY(bh::evaluate(c, p));
        c->have_acc = true;
    }
    for (int s = 0; s < nsteps; ++s) {
        c->early_now = s == nsteps - 1;  // only the last step's evaluation counts
        if (c->tune.graph && c->have_lists && c->k_eval % c->prm.rebuild_every != 0) {
            BH_TRY(bh::graph_reuse_step(c, p));
            continue;
        }
        // a list capacity needs the eager build's exact sizes
        if (c->tune.graph == 1 && c->have_lists && c->prm.list_capacity == 0) {
            BH_TRY(bh::graph_rebuild_step(c, p));
            continue;
        }
        BH_TRY(bh::stage_kick_drift(c, p, 0.5 * dt, dt));
        BH_TRY(bh::evaluate(c, p));
        BH_TRY(bh::stage_kick(c, p, 0.5 * dt));
    }
    return BH_OK;
}

int bh_set_tuning(bh_ctx* ctx, const bh_tuning* t) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    BH_TRY(bh::check_tuning(c, t));
    const bool reorder = t->chunk != c->tune.chunk || t->order_by_cost != c->tune.order_by_cost ||
                         t->order_window != c->tune.order_window;
    bh::apply_tuning(c, t);
    if (reorder && c->have_lists && c->prm.precision == BH_PREC_FP32) BH_TRY(bh::build_order32(c));
    return BH_OK;
}

int bh_get_tuning(bh_ctx* ctx, bh_tuning* t) {
    Ctx* c = (Ctx*)ctx;
    if (!c || !t) return BH_E_INVAL;
    bh::read_tuning(c, t);
    return BH_OK;
}

int bh_autotune(bh_ctx* ctx, bh_particles* p, double* best_ms) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    return bh::autotune(c, p, best_ms);
}

int bh_get_diagnostics(bh_ctx* ctx, const bh_particles* p, bh_diagnostics* out) {
    Ctx* c = (Ctx*)ctx;
    if (!c || !out) return BH_E_INVAL;
    BH_TRY(bh::check_particles(c, p, true));
    double s[11];
    BH_TRY(bh::stage_diagnostics(c, p, s));
    out->mass = s[0];
    for (int a = 0; a < 3; ++a) {
        out->momentum[a] = s[1 + a];
        out->angular_momentum[a] = s[4 + a];
    }
    out->kinetic = s[7];
    out->potential_central = s[8];
    out->contact_candidates = -1;
    out->contacts = -1;
    if (c->contact_stats) {
        unsigned long long h[3];
        BH_CUDA(c, cudaMemcpyAsync(h, c->d_small + 16, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
        out->contact_candidates = (int64_t)h[0];
        out->contacts = (int64_t)(h[2] / 2);
    }
    return bh::read_status(c);
}

int bh_compute_potential(bh_ctx* ctx, const bh_particles* p, double* phi, double* W) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_lists) return bh::fail(c, BH_E_STATE, "bh_compute_potential needs lists (call bh_make_lists)");
    BH_TRY(bh::check_particles(c, p, false));
    if (p->n != c->n) return bh::fail(c, BH_E_INVAL, "particle count changed since the tree was built");
    BH_TRY(bh::stage_potential(c, p, phi, W));
    return W ? bh::read_status(c) : BH_OK;
}

int bh_get_balance(bh_ctx* ctx, double* busy_fraction) {
    Ctx* c = (Ctx*)ctx;
    if (!c || !busy_fraction) return BH_E_INVAL;
    if (c->warp_time_n <= 0 || !c->warp_time.p) return bh::fail(c, BH_E_STATE, "no timed persistent force launch");
    std::vector<unsigned long long> t(2 * (size_t)c->warp_time_n);
    BH_CUDA(c, cudaMemcpyAsync(t.data(), c->warp_time.p, t.size() * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, c->stream));
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    unsigned long long t0 = ~0ull, t1 = 0;
    double busy = 0.0;
    for (int64_t w = 0; w < c->warp_time_n; ++w) {
        t0 = std::min(t0, t[2 * w]);
        t1 = std::max(t1, t[2 * w + 1]);
        busy += (double)(t[2 * w + 1] - t[2 * w]);
    }
    *busy_fraction = t1 > t0 ? busy / ((double)c->warp_time_n * (double)(t1 - t0)) : 1.0;
    return BH_OK;
}

int bh_step_host(bh_ctx* ctx, bh_particles* h, int nsteps) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    BH_TRY(bh::check_particles(c, h, true));
    if (!h->id) return bh::fail(c, BH_E_INVAL, "id must be set");
    const int64_t n = h->n;
    BH_TRY(bh::grow(c, c->hbuf, (size_t)n * 10, "host-step particle buffers"));
    BH_TRY(bh::grow(c, c->hid, (size_t)n, "host-step ids"));
    double* b = c->hbuf.p;
    bh_particles d;
    d.x = b; d.y = b + n; d.z = b + 2 * n; d.vx = b + 3 * n; d.vy = b + 4 * n; d.vz = b + 5 * n;
    d.m = b + 6 * n; d.ax = b + 7 * n; d.ay = b + 8 * n; d.az = b + 9 * n; d.id = c->hid.p; d.n = n;
    double* hs[10] = {h->x, h->y, h->z, h->vx, h->vy, h->vz, h->m, h->ax, h->ay, h->az};
    double* ds[10] = {d.x, d.y, d.z, d.vx, d.vy, d.vz, d.m, d.ax, d.ay, d.az};
    // Only list-constructing evaluations reorder the particles.  When this
    // call has none, the ids are not needed on the device and neither ids
    // nor masses change, so they are not copied (the caller's copies stay
    // current; a later list build copies the ids in before reordering them).
    bool reorder = !c->have_lists || !c->have_acc;
    for (int64_t k = c->k_eval; !reorder && k < c->k_eval + nsteps; ++k) reorder = k % c->prm.rebuild_every == 0;
    const int ncopy = c->have_acc ? 10 : 7;
    for (int a = 0; a < ncopy; ++a)
        BH_CUDA(c, cudaMemcpyAsync(ds[a], hs[a], n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    c->h2d_bytes += (int64_t)ncopy * n * (int64_t)sizeof(double);
    if (reorder) {
        BH_CUDA(c, cudaMemcpyAsync(d.id, h->id, n * sizeof(int64_t), cudaMemcpyHostToDevice, c->stream));
        c->h2d_bytes += n * (int64_t)sizeof(int64_t);
    }
    if (!c->copy_stream) BH_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
    if (!c->pos_event) BH_CUDA(c, cudaEventCreateWithFlags(&c->pos_event, cudaEventDisableTiming));
    c->want_pos_event = true;
    c->pos_event_recorded = false;
    c->early_dst = h;
    c->early_src = &d;
    c->early_ids = reorder;
    // From here on the copy stream may hold copies into the caller's host
    // arrays: every return waits for them, so none is still writing after
    // the call has returned (with an error or not).
    struct CopyStreamGuard {
        cudaStream_t s;
        ~CopyStreamGuard() {
            if (s) cudaStreamSynchronize(s);
        }
    } guard{c->copy_stream};
    const int rc = bh_step(ctx, &d, nsteps);
    c->want_pos_event = false;
    c->early_now = false;
    c->early_dst = c->early_src = nullptr;
    BH_TRY(rc);
    // positions, masses and ids: their copy back was enqueued on the second
    // stream by the last evaluation as soon as they were final (so it ran
    // with the force kernel); velocities and accelerations follow the final
    // kick.  A step run as a graph has no such point: everything after it.
    const bool early = c->pos_event_recorded;
    const int late_from = early ? 3 : 0;
    int64_t out_bytes = early ? (reorder ? 4 : 3) * n * (int64_t)sizeof(double) +
                                    (reorder ? n * (int64_t)sizeof(int64_t) : 0)
                              : 0;
    for (int a = late_from; a < 10; ++a) {
        if ((early || !reorder) && a == 6) continue;  // masses: copied early, or unchanged
        BH_CUDA(c, cudaMemcpyAsync(hs[a], ds[a], n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        out_bytes += n * (int64_t)sizeof(double);
    }
    if (!early && reorder) {
        BH_CUDA(c, cudaMemcpyAsync(h->id, d.id, n * sizeof(int64_t), cudaMemcpyDeviceToHost, c->stream));
        out_bytes += n * (int64_t)sizeof(int64_t);
    }
    c->d2h_bytes += out_bytes;
    if (early) BH_CUDA(c, cudaStreamSynchronize(c->copy_stream));
    guard.s = nullptr;  // waited for above
    return bh_sync(ctx);
}

int bh_sync(bh_ctx* ctx) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    return bh::read_status(c);
}

int bh_get_sizes(bh_ctx* ctx, int64_t* n_nodes, int64_t* n_groups, int64_t* n_pp, int64_t* n_pc, int64_t* n_jj) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (n_nodes) *n_nodes = c->have_tree ? c->n_nodes : 0;
    if (n_groups) *n_groups = c->have_tree ? c->n_groups : 0;
    if (n_pp) *n_pp = c->have_lists ? c->n_pp : c->list_overflowed ? c->need_pp : 0;
    if (n_pc) *n_pc = c->have_lists ? c->n_pc : c->list_overflowed ? c->need_pc : 0;
    if (n_jj) *n_jj = c->have_lists ? c->n_jj : c->list_overflowed ? c->need_jj : 0;
    return BH_OK;
}

#define BH_D2H(c, dst, src, bytes)                                                                   \
    do {                                                                                             \
        if (dst) BH_CUDA(c, cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyDeviceToHost, c->stream)); \
    } while (0)

int bh_get_keys(bh_ctx* ctx, uint64_t* keys, uint32_t* perm) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_tree) return bh::fail(c, BH_E_STATE, "no tree");
    BH_D2H(c, keys, c->key[c->key_cur].p, c->n * sizeof(uint64_t));
    BH_D2H(c, perm, c->idx[c->key_cur].p, c->n * sizeof(uint32_t));
    return bh::read_status(c);
}

int bh_get_root(bh_ctx* ctx, double* lo3, double* L) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_tree) return bh::fail(c, BH_E_STATE, "no tree");
    std::vector<double> box(8 * (size_t)c->n_patches);
    BH_CUDA(c, cudaMemcpyAsync(box.data(), c->d_box, box.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < c->n_patches; ++q) {
        if (lo3)
            for (int a = 0; a < 3; ++a) lo3[3 * q + a] = box[8 * q + a];
        if (L) L[q] = box[8 * q + 3];
    }
    return bh::read_status(c);
}

int bh_get_tree(bh_ctx* ctx, uint8_t* level, uint32_t* begin, uint32_t* end, int32_t* parent,
                int32_t* first_child, uint8_t* nchild, uint32_t* qlo3, uint32_t* qhi3) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_tree) return bh::fail(c, BH_E_STATE, "no tree");
    const size_t nn = (size_t)c->n_nodes;
    BH_D2H(c, level, c->level.p, nn);
    BH_D2H(c, begin, c->begin.p, nn * 4);
    BH_D2H(c, end, c->end.p, nn * 4);
    BH_D2H(c, parent, c->parent.p, nn * 4);
    BH_D2H(c, first_child, c->first_child.p, nn * 4);
    BH_D2H(c, nchild, c->nchild.p, nn);
    BH_D2H(c, qlo3, c->qlo.p, nn * 12);
    BH_D2H(c, qhi3, c->qhi.p, nn * 12);
    return bh::read_status(c);
}

int bh_get_moments(bh_ctx* ctx, double* M, double* c3, double* Q6) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_tree) return bh::fail(c, BH_E_STATE, "no tree");
    const size_t nn = (size_t)c->n_nodes;
    if (c->prm.precision == BH_PREC_FP32) {
        // the FP32 path keeps FP32 records: centre as hi + lo, M, Q (traceless)
        std::vector<float4> rec(nn * 3);
        BH_CUDA(c, cudaMemcpyAsync(rec.data(), c->cell32.p, nn * 3 * sizeof(float4), cudaMemcpyDeviceToHost,
                                   c->stream));
        BH_TRY(bh::read_status(c));
        for (size_t k = 0; k < nn; ++k) {
            const float4 h = rec[3 * k], l = rec[3 * k + 1], u = rec[3 * k + 2];
            if (M) M[k] = h.w;
            if (c3) {
                c3[k] = (double)h.x + (double)l.x;
                c3[nn + k] = (double)h.y + (double)l.y;
                c3[2 * nn + k] = (double)h.z + (double)l.z;
            }
            if (Q6) {
                const double q[6] = {l.w, u.z, -((double)l.w + (double)u.z), u.x, u.y, u.w};
                for (int a = 0; a < 6; ++a) Q6[6 * k + a] = q[a];
            }
        }
        return BH_OK;
    }
    BH_D2H(c, M, c->M.p, nn * 8);
    if (c3) {
        double* cys = c3 + nn;
        double* czs = c3 + 2 * nn;
        BH_CUDA(c, cudaMemcpyAsync(c3, c->cx.p, nn * 8, cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaMemcpyAsync(cys, c->cy.p, nn * 8, cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaMemcpyAsync(czs, c->cz.p, nn * 8, cudaMemcpyDeviceToHost, c->stream));
    }
    BH_D2H(c, Q6, c->Q.p, nn * 48);
    return bh::read_status(c);
}

int bh_get_groups(bh_ctx* ctx, int32_t* group_nodes) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_tree) return bh::fail(c, BH_E_STATE, "no tree");
    BH_D2H(c, group_nodes, c->groups.p, (size_t)c->n_groups * 4);
    return bh::read_status(c);
}

int bh_get_lists(bh_ctx* ctx, int64_t* pp_off, int32_t* pp_ids, int64_t* pc_off, int32_t* pc_ids) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (!c->have_lists) return bh::fail(c, BH_E_STATE, "no lists");
    const size_t ng = (size_t)c->n_groups;
    BH_D2H(c, pp_off, c->cnt_p.p, (ng + 1) * 8);
    BH_D2H(c, pp_ids, c->P.p, (size_t)c->n_pp * 4);
    BH_D2H(c, pc_off, c->cnt_c.p, (ng + 1) * 8);
    BH_D2H(c, pc_ids, c->C.p, (size_t)c->n_pc * 4);
    return bh::read_status(c);
}

int bh_get_counters(bh_ctx* ctx, bh_counters* out) {
    Ctx* c = (Ctx*)ctx;
    if (!c || !out) return BH_E_INVAL;
    out->n_groups = c->n_groups;
    out->n_pp = c->n_int_pp;
    out->n_pc = c->n_int_pc;
    out->n_evals = c->evals_since_build;
    out->n_rebuilds = c->n_rebuilds;
    out->n_launches = c->n_launches;
    out->n_contacts = c->n_contacts;
    out->n_pp_far = c->n_int_pp_far;
    out->n_one_walk_builds = c->n_one_walk_builds;
    out->n_h2d_bytes = c->h2d_bytes;
    out->n_d2h_bytes = c->d2h_bytes;
    if (c->refine_pending) {  // an evaluation without a read-back since: read its count now
        unsigned long long nr = 0;
        BH_CUDA(c, cudaMemcpyAsync(&nr, c->d_small + 20, sizeof(nr), cudaMemcpyDeviceToHost, c->stream));
        BH_CUDA(c, cudaStreamSynchronize(c->stream));
        c->n_refined = (int64_t)nr;
        c->refine_pending = false;
    }
    out->n_refined = c->n_refined;
    out->n_graph_builds = c->n_graph_builds;
    out->n_graph_build_redos = c->n_graph_build_redos;
    out->n_graph_captures = c->n_graph_captures;
    BH_TRY(bh::read_stage_events(c, false));
    for (int s = 0; s < BH_N_STAGES; ++s) {
        out->stage_ms[s] = c->stage_ms[s];
        out->stage_calls[s] = c->stage_calls[s];
    }
    return BH_OK;
}

int bh_set_list_capacity(bh_ctx* ctx, int64_t entries) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    if (entries < 0) return bh::fail(c, BH_E_INVAL, "list capacity must be >= 0");
    c->prm.list_capacity = entries;
    return BH_OK;
}

int bh_set_timing(bh_ctx* ctx, int enable) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    c->timing = enable != 0;
    return BH_OK;
}

int bh_get_timing(bh_ctx* ctx, double* force_ms, int64_t* force_launches, int reset) {
    Ctx* c = (Ctx*)ctx;
    if (!c) return BH_E_INVAL;
    BH_CUDA(c, cudaStreamSynchronize(c->stream));
    double total = 0.0;
    for (auto& pr : c->ev_force) {
        float ms = 0.f;
        BH_CUDA(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
        total += ms;
    }
    if (force_ms) *force_ms = total;
    if (force_launches) *force_launches = (int64_t)c->ev_force.size();
    if (reset) {
        for (auto& pr : c->ev_force) {
            c->ev_pool.push_back(pr.first);
            c->ev_pool.push_back(pr.second);
        }
        c->ev_force.clear();
        BH_TRY(bh::read_stage_events(c, true));
        for (int s = 0; s < BH_N_STAGES; ++s) {
            c->stage_ms[s] = 0.0;
            c->stage_calls[s] = 0;
        }
    }
    return BH_OK;
}

}  // extern "C"
