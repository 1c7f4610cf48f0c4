// server.cu -- the serving form of the voter: continuous batching of vote
// requests (ft_server_create / ft_submit / ft_poll).
//
// Requests are admitted against a device-memory budget: each one holds
// (R+1) * n * sizeof(dtype) bytes of resident replicas and output until its
// result is collected.  A worker thread packs the admitted requests that are
// waiting into the next batch (up to max_slots), lays the batch out for the
// persistent batched kernels and launches it on one of `streams` CUDA
// streams, so that a new batch starts while earlier ones are still on the
// device.  The worker detects completed batches by polling an event per batch
// (spinning while batches are in flight, and for a short while after, before
// it sleeps), marks their requests done, and ft_poll waits for that with a
// bound, as the paper's runtime bounds the wait for a task by a timeout
// (Sec. IV.C).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "batched.h"
#include "ftvote.h"
#include "resident.h"
#include "runtime.h"

namespace {

double now_us()
{
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
    ftv::TaskArgs args;
    ft_stats *user_stats = nullptr;
    unsigned long long bytes = 0;
    double submit_us = 0, done_us = 0, launch_us = 0, launched_us = 0;
    int status = FT_EAGAIN;
    bool done = false;
    ft_stats result;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;        // recorded after the batch's kernels
    uint8_t *dev = nullptr;            // batch layout (device)
    size_t dev_cap = 0;
    uint8_t *host = nullptr;           // batch layout staging (pinned)
    size_t host_cap = 0;
    double launched_at = 0.0;          // worker clock when the batch began to launch
    double launch_done_at = 0.0;       // and when its launch calls had returned
    ft_stats *host_stats = nullptr;    // pinned copy of the batch's statistics, read once the event completes
    ft_stats *host_stats_dev = nullptr;   // the same memory as the device addresses it
    ft_stats **dev_user = nullptr;     // caller stats pointers (scatter targets)
    ft_stats **host_user = nullptr;    // pinned
    int cap = 0;                       // requests per batch
    bool busy = false;
    int status = FT_OK;
    std::vector<unsigned long long> tickets;
    ftv::BatchLayout layout;
    std::vector<ftv::GroupDev> gd;
    // small batches (at most kSmallTasks requests, no caller statistics
    // pointers) travel in the kernel parameters; their tile and done counters
    // and statistics live here, left reset by each group kernel's last CTA
    uint8_t *small_area = nullptr;
    unsigned long long *small_cnt = nullptr;   // 2 per group: tile counter, done counter
    ft_stats *small_stats = nullptr;           // one per request
    unsigned long long *small_tiles = nullptr; // per request of a small batch: its tiles voted so far
    bool small_dirty = true;                   // re-initialise before the next small batch
    bool last_small = false;                   // the batch in flight took the small path
    // Completion request by request: the kernels write the batch's sequence
    // number to flags[i] (pinned, host-mapped) once request i's statistics
    // are in host_stats[i], so a request is done as soon as its own tiles are
    // voted, not when its whole batch is.  The slot itself is free for the
    // next batch only once the batch's event has completed.
    unsigned long long *flags = nullptr;
    unsigned long long *flags_dev = nullptr;
    unsigned long long seq = 0;
    bool per_req = false;                      // the batch in flight completes request by request
    std::vector<char> req_done;
    size_t ndone = 0;
    double last_check = 0.0;                   // last event query while requests were outstanding
    bool ended = false;                        // the event was seen complete
    // a batch's (kind, R) groups after the first run on these streams, forked
    // from and joined back into `stream` with events
    cudaStream_t aux[3] = {};
    cudaEvent_t forked = nullptr, joined[3] = {};
};

constexpr int kAuxStreams = 3;

// The stream of a batch's group gi: the slot's own for the first, then the
// auxiliary streams in turn.  With an upload, fork() records `forked` right
// after it (before any group is launched) and the first use of an auxiliary
// stream in the batch waits for it; a small batch has nothing to wait for.
struct GroupStreams {
    Slot &sl;
    bool forked = false;
    bool used[kAuxStreams] = {};
    cudaError_t fork()
    {
        forked = true;
        return cudaEventRecord(sl.forked, sl.stream);
    }
    cudaStream_t get(int gi, cudaError_t *e)
    {
        *e = cudaSuccess;
        if (gi == 0) return sl.stream;
        const int a = (gi - 1) % kAuxStreams;
        if (!used[a]) {
            if (forked) *e = cudaStreamWaitEvent(sl.aux[a], sl.forked, 0);
            used[a] = true;
        }
        return sl.aux[a];
    }
    // the slot's stream waits for every auxiliary stream this batch used
    cudaError_t join()
    {
        cudaError_t e = cudaSuccess;
        for (int a = 0; a < kAuxStreams && e == cudaSuccess; ++a)
            if (used[a] && (e = cudaEventRecord(sl.joined[a], sl.aux[a])) == cudaSuccess)
                e = cudaStreamWaitEvent(sl.stream, sl.joined[a], 0);
        return e;
    }
};

// the small-batch area: 2 counters per group, then a tile count per request
// (all zero), then the requests' statistics
constexpr size_t kSmallCntBytes = 3 * ftv::kSmallTasks * sizeof(unsigned long long);
constexpr size_t kSmallAreaBytes = kSmallCntBytes + ftv::kSmallTasks * sizeof(ft_stats);

ft_stats initial_stats()
{
    ft_stats st;
    for (int r = 0; r < FT_MAX_R; ++r) {
        st.mismatch[r] = 0;
        st.first_mismatch[r] = -1;
    }
    st.no_majority = 0;
    st.first_no_majority = -1;
    return st;
}

// The resident mode (ft_server_config.resident): no batches and no launch per
// request.  The worker hands each request to a free device slot through a
// host-mapped mailbox and keeps the resident kernel (resident.cu) running
// while any slot is busy; the kernel writes each request's statistics and
// flag to host-mapped memory when its last tile is voted.
struct Resident {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;          // recorded after each launch: the kernel has left
    uint8_t *dev = nullptr;              // device block: slots, counters, statistics
    uint8_t *host = nullptr;             // host-mapped block: mailboxes, flags, statistics copies
    ftv::ResDev g{};                     // the kernel's view of both
    ftv::ResMail *mail = nullptr;        // host views of the host-mapped block
    unsigned long long *mail_gen = nullptr;
    unsigned int *quit = nullptr;
    unsigned int *error = nullptr;
    ft_stats *stats_out = nullptr;
    unsigned long long *flags = nullptr;
    unsigned long long slot_gen[ftv::kResSlots] = {};     // generation on slot j, 0 = free
    unsigned long long slot_ticket[ftv::kResSlots] = {};
    double slot_sent[ftv::kResSlots] = {};
    unsigned long long gen = 0;          // last generation handed out
    int voting_warps = 1;
    int max_ctas = 0;                    // grid cap (the shared mode: the SMs the batches leave free)
    bool running = false;                // launched, not yet seen to have left
    double last_query = 0.0;
    int failed = FT_OK;                  // the kernel reported an error or a launch failed
    unsigned long long launches = 0;
};

}  // namespace

struct ft_server {
    ft_server_config cfg{};
    bool auto_tile = false;            // tile size chosen per batch (configured as 0)
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work;   // worker: new requests, a free slot, stop
    std::condition_variable cv_done;   // pollers: a request completed
    std::deque<unsigned long long> pending;
    std::unordered_map<unsigned long long, Request> reqs;
    unsigned long long next_ticket = 1;
    unsigned long long inflight_bytes = 0;
    int inflight = 0;
    bool stop = false;
    bool paused = false;
    std::vector<Slot> slots;
    std::thread worker;
    unsigned long long batch_seq = 0;  // sequence number of the last batch launched (worker only)
    // counters reported by ft_server_info
    unsigned long long batches = 0, batched_requests = 0, completed = 0;
    int busy_now = 0, busy_max = 0;
    double launch_host_us = 0.0, batch_span_us = 0.0, queue_us = 0.0;
    // bumped (under the lock) whenever there is something new for the worker:
    // an admitted request, a pause change or stop
    std::atomic<unsigned long long> version{0};
    bool resident = false;             // resident-kernel memory allocated (resident = 1 or 2)
    bool hybrid = false;               // resident = 2: small requests to the resident kernel
    Resident res;
};

namespace {

// Request i of slot si is done with `status` (lock held).
void complete_request(ft_server *s, Slot &sl, size_t i, double t, int status)
{
    sl.req_done[i] = 1;
    sl.ndone += 1;
    s->completed += 1;
    auto it = s->reqs.find(sl.tickets[i]);
    if (it == s->reqs.end()) return;
    Request &r = it->second;
    r.result = sl.host_stats[i];
    r.status = status;
    r.done = true;
    r.done_us = t;
    r.launch_us = sl.launched_at;
    r.launched_us = sl.launch_done_at;
}

// The batch of slot si has left the device: its remaining requests are done
// with the batch's status, and the slot takes the next batch (lock held).
void complete_slot(ft_server *s, int si, double t)
{
    Slot &sl = s->slots[si];
    for (size_t i = 0; i < sl.tickets.size(); ++i)
        if (!sl.req_done[i]) complete_request(s, sl, i, t, sl.status);
    if (sl.last_small && sl.status != FT_OK) sl.small_dirty = true;
    s->batch_span_us += t - sl.launched_at;
    sl.tickets.clear();
    sl.busy = false;
    s->busy_now -= 1;
    s->cv_done.notify_all();
}

// Requests of a batch with per-request completion whose flag is set
// (lock held); returns how many.
size_t reap_flags(ft_server *s, Slot &sl, double t)
{
    size_t k = 0;
    for (size_t i = 0; i < sl.tickets.size(); ++i)
        if (!sl.req_done[i] && __atomic_load_n(&sl.flags[i], __ATOMIC_ACQUIRE) == sl.seq) {
            complete_request(s, sl, i, t, FT_OK);
            ++k;
        }
    return k;
}

// While requests of a batch are outstanding its event is queried at most this
// often (µs): a batch whose kernels ended without flagging a request (a CUDA
// failure) completes through it.
constexpr double kEventCheckUs = 100.0;

// Completions of slot si (lock held).  Returns true when something changed.
bool reap_slot(ft_server *s, int si)
{
    Slot &sl = s->slots[si];
    const double t = now_us();
    bool changed = false;
    if (sl.per_req) {
        if (reap_flags(s, sl, t)) {
            changed = true;
            s->cv_done.notify_all();
        }
        if (sl.ndone < sl.tickets.size() && !sl.ended) {
            if (t - sl.last_check < kEventCheckUs) return changed;
            sl.last_check = t;
        }
    }
    const cudaError_t q = cudaEventQuery(sl.done);
    if (q == cudaErrorNotReady) return changed;
    if (q != cudaSuccess) sl.status = ftv::cuda_fail(q);
    if (sl.per_req && sl.status == FT_OK) {
        // the kernels have ended: every flag they wrote is visible
        reap_flags(s, sl, t);
        // a request that the kernels left unflagged did not complete
        if (sl.ndone < sl.tickets.size()) sl.status = FT_ECUDA;
    }
    complete_slot(s, si, t);
    return true;
}

// Whether slot si has anything to reap (no lock: only the worker changes a
// busy slot's fields).
bool slot_progress(Slot &sl)
{
    if (sl.per_req) {
        for (size_t i = 0; i < sl.tickets.size(); ++i)
            if (!sl.req_done[i] && __atomic_load_n(&sl.flags[i], __ATOMIC_ACQUIRE) == sl.seq) return true;
        if (sl.ndone < sl.tickets.size()) {
            const double t = now_us();
            if (t - sl.last_check < kEventCheckUs) return false;
            sl.last_check = t;
        }
    }
    if (cudaEventQuery(sl.done) == cudaErrorNotReady) return false;
    sl.ended = true;   // reap_slot then completes the batch without waiting for its next check
    return true;
}

int grow_slot(Slot &sl, size_t layout_bytes, int nreq)
{
    cudaError_t e;
    if (layout_bytes > sl.dev_cap) {
        if (sl.dev) cudaFree(sl.dev);
        if (sl.host) cudaFreeHost(sl.host);
        sl.dev = sl.host = nullptr;
        sl.dev_cap = sl.host_cap = 0;
        const size_t cap = layout_bytes + layout_bytes / 2;
        if ((e = cudaMalloc(&sl.dev, cap)) != cudaSuccess) return ftv::cuda_fail(e);
        if ((e = cudaMallocHost(&sl.host, cap)) != cudaSuccess) return ftv::cuda_fail(e);
        sl.dev_cap = sl.host_cap = cap;
    }
    if (nreq > sl.cap) {
        if (sl.host_stats) cudaFreeHost(sl.host_stats);
        if (sl.flags) cudaFreeHost(sl.flags);
        if (sl.dev_user) cudaFree(sl.dev_user);
        if (sl.host_user) cudaFreeHost(sl.host_user);
        sl.host_stats = nullptr;
        sl.flags = nullptr;
        sl.dev_user = sl.host_user = nullptr;
        sl.cap = 0;
        if ((e = cudaMallocHost(&sl.host_stats, sizeof(ft_stats) * nreq)) != cudaSuccess) return ftv::cuda_fail(e);
        if ((e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&sl.host_stats_dev), sl.host_stats, 0)) !=
            cudaSuccess)
            return ftv::cuda_fail(e);
        if ((e = cudaMallocHost(&sl.flags, sizeof(unsigned long long) * nreq)) != cudaSuccess) return ftv::cuda_fail(e);
        std::memset(sl.flags, 0, sizeof(unsigned long long) * nreq);   // batch sequence numbers start at 1
        if ((e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&sl.flags_dev), sl.flags, 0)) != cudaSuccess)
            return ftv::cuda_fail(e);
        if ((e = cudaMalloc(&sl.dev_user, sizeof(ft_stats *) * nreq)) != cudaSuccess) return ftv::cuda_fail(e);
        if ((e = cudaMallocHost(&sl.host_user, sizeof(ft_stats *) * nreq)) != cudaSuccess) return ftv::cuda_fail(e);
        sl.cap = nreq;
    }
    return FT_OK;
}

// SMs that no batch's kernels may fill while the server has several streams:
// a voter CTA holds a whole SM (its CRC tables), so without them a batch that
// arrives behind a large one waits for all of the large one's CTAs to exit.
// Replays of the 20k and 60k requests/s streams, continuous batching, 3
// streams: none reserved p99 0.36 / 1.11 ms, 16 SMs 0.29 / 0.92 ms, and 32 SMs
// 0.22 / 0.64 ms (16: 0.24 / 0.87 ms in the same run) once the worker polled
// without holding the server's lock; p50 within the runs' spread.
// ft_server_config.reserved_sms overrides it.
constexpr int kReservedSms = 32;

int batch_max_ctas(const ft_server *s, const ftv::TaskArgs &a)
{
    const int reserve = s->cfg.reserved_sms == 0 ? kReservedSms : s->cfg.reserved_sms;
    if (s->slots.size() < 2 || reserve <= 0) return 0;
    int sms = 0, per_sm = 0;
    if (ftv::group_occupancy(a.kind, a.R, &sms, &per_sm) != FT_OK) return 0;
    return sms > reserve ? (sms - reserve) * per_sm : per_sm;
}

// Warps per CTA of a group of `tiles` work tiles that may use `max_ctas` CTAs
// (0 = one per SM): a group too small to give every CTA 16 tiles runs 8-warp
// CTAs, which spreads it over twice as many SMs (for the single-task voter 8
// warps measured 10.0 against 12.3 us on 3 x 1M f32 and 3 x 256K f32); a
// larger one keeps 16 warps per SM for bandwidth.
int group_warps(const ftv::TaskArgs &a, unsigned long long tiles, int max_ctas)
{
    int cap = max_ctas;
    if (cap <= 0) {
        int sms = 0, per_sm = 0;
        if (ftv::group_occupancy(a.kind, a.R, &sms, &per_sm) != FT_OK) return ftv::kBatchWarps;
        cap = sms * per_sm;
    }
    return tiles < (unsigned long long)cap * ftv::kBatchWarps ? 8 : ftv::kBatchWarps;
}

// A small batch: its (kind, R) groups are launched with their tasks in the
// kernel parameters, so nothing is uploaded, and each request's statistics
// come back through the warp that votes its last tile, with its flag.  The
// requests with skip[i] set are left out (they vote on their own).  Group g
// runs on gs's stream g; *launched returns how many streams were used.  The
// caller joins gs.
int launch_small_batch(Slot &sl, GroupStreams &gs, const std::vector<ftv::TaskArgs> &args, const bool *skip,
                       int tile, int max_ctas, int *launched_out)
{
    const int n_all = (int)args.size();
    cudaError_t e;
    *launched_out = 0;
    if (sl.small_dirty) {
        // first use, or a failed batch may have left counters or statistics set
        uint8_t init[kSmallAreaBytes];
        std::memset(init, 0, kSmallCntBytes);
        const ft_stats st = initial_stats();
        for (int i = 0; i < ftv::kSmallTasks; ++i) std::memcpy(init + kSmallCntBytes + i * sizeof(ft_stats), &st, sizeof st);
        if ((e = cudaMemcpyAsync(sl.small_area, init, kSmallAreaBytes, cudaMemcpyHostToDevice, sl.stream)) !=
                cudaSuccess ||
            (e = cudaStreamSynchronize(sl.stream)) != cudaSuccess)
            return ftv::cuda_fail(e);
        sl.small_dirty = false;
    }
    int order[ftv::kSmallTasks];
    int n = 0;
    for (int i = 0; i < n_all; ++i)
        if (!skip[i]) order[n++] = i;
    std::stable_sort(order, order + n, [&](int x, int y) {
        return std::make_pair(args[x].kind, args[x].R) < std::make_pair(args[y].kind, args[y].R);
    });
    ftv::SmallGroup g;
    int gi = 0, launched = 0;
    for (int i = 0; i < n; ++gi) {
        std::memset(&g, 0, sizeof g);
        g.kind = args[order[i]].kind;
        g.R = args[order[i]].R;
        g.tile_blocks = tile;
        for (; i < n && args[order[i]].kind == g.kind && args[order[i]].R == g.R; ++i) {
            ftv::TaskArgs a = args[order[i]];
            a.stats = sl.small_stats + order[i];
            g.tile_first[g.ntasks] = g.total_tiles;
            g.total_tiles += (a.nfull + (a.tail_bytes ? 1 : 0) + tile - 1) / tile;
            g.tasks[g.ntasks++] = a;
        }
        g.warps = group_warps(g.tasks[0], g.total_tiles, max_ctas);
        g.counter = sl.small_cnt + 2 * gi;
        g.done_ctas = sl.small_cnt + 2 * gi + 1;
        g.stats_base = sl.small_stats;
        g.stats_out = sl.host_stats_dev;
        g.tiles_done = sl.small_tiles;
        g.flag_out = sl.flags_dev;
        g.seq = sl.seq;
        // only empty requests: no kernel (launch_slot has completed them)
        if (g.total_tiles == 0) continue;
        cudaStream_t st = gs.get(launched++, &e);
        *launched_out = launched;
        const int rc = e == cudaSuccess ? ftv::launch_small_group(g, st, max_ctas) : ftv::cuda_fail(e);
        if (rc != FT_OK) {
            sl.small_dirty = true;
            return rc;
        }
    }
    return FT_OK;
}

// Request bytes from which a request of a small batch votes on its own, as a
// single vote through the single-task voter, instead of in the batch's group
// kernel: (R+1) x its bytes, 64 MiB (10 us of HBM time).  It then gets the
// single-task shapes (for f32 R = 3 the prefetching 12-warp one), runs on a
// stream of its own beside the batch's small requests, and does not wait for
// them.
constexpr unsigned long long kOwnVoteBytes = 64ull << 20;

unsigned long long task_bytes(const ftv::TaskArgs &a)
{
    return (unsigned long long)(a.R + 1) * (a.nfull * FT_BLOCK_BYTES + a.tail_bytes);
}

// Launch the requests `tickets` as one batch on slot `si` (lock not held).
// Without caller statistics pointers each request completes on its own (its
// flag); with them, the statistics are scattered to the callers' buffers after
// the group kernels and the batch completes as a whole (its event).
int launch_slot(ft_server *s, int si, std::vector<ftv::TaskArgs> &args, bool any_user)
{
    Slot &sl = s->slots[si];
    const int n = (int)args.size();
    for (int i = 0; i < n; ++i) args[i].stats = nullptr;   // set below, after growing
    int rc = grow_slot(sl, 0, n);
    if (rc != FT_OK) return rc;
    // empty requests have nothing to vote: done at launch, statistics initial
    for (int i = 0; i < n; ++i)
        if (args[i].n == 0) {
            sl.host_stats[i] = initial_stats();
            __atomic_store_n(&sl.flags[i], sl.seq, __ATOMIC_RELEASE);
        }
    int tile = s->cfg.tile_blocks;
    if (s->auto_tile) {
        unsigned long long total = 0;
        for (const ftv::TaskArgs &a : args) total += a.nfull + (a.tail_bytes ? 1 : 0);
        int sms = 0, per_sm = 0;
        if ((rc = ftv::group_occupancy(args[0].kind, args[0].R, &sms, &per_sm)) != FT_OK) return rc;
        // each of the batches in flight at once gets about its share of a wave
        tile = ftv::auto_tile_blocks(total, (unsigned long long)sms * per_sm * ftv::kBatchWarps / s->slots.size());
    }
    const int max_ctas = batch_max_ctas(s, args[0]);
    sl.last_small = n <= ftv::kSmallTasks && !any_user;
    if (sl.last_small) {
        // A lone request, and each large one, votes on its own through the
        // single-task voter (its statistics through one of the voter's slots,
        // copied straight into this slot's pinned array, then its flag): the
        // single-task shapes take 3.1 us less kernel time than the batched
        // kernel at 16 KiB per replica, and for large f32 R = 3 votes the
        // prefetching 12-warp shape.  If the voter's slots run out, every
        // request goes through the small-batch kernels.
        bool own[ftv::kSmallTasks] = {};
        int vslot[ftv::kSmallTasks];
        for (int i = 0; i < n; ++i) {
            if (args[i].n == 0 || (n > 1 && task_bytes(args[i]) < kOwnVoteBytes)) continue;
            if ((vslot[i] = ftv::reserve_vote_slot()) < 0) {
                for (int k = 0; k < i; ++k)
                    if (own[k]) ftv::release_vote_slot(vslot[k]);
                std::fill(own, own + n, false);
                break;
            }
            own[i] = true;
        }
        bool any_small = false;
        for (int i = 0; i < n; ++i) any_small |= !own[i] && args[i].n > 0;
        GroupStreams gs{sl};
        int used = 0;
        if (any_small) rc = launch_small_batch(sl, gs, args, own, tile, max_ctas, &used);
        else sl.last_small = false;   // the small-batch area is not used
        // the requests voting on their own one after another (smallest first),
        // on the stream after the small requests' groups
        cudaStream_t st = nullptr;
        for (int i = 0; i < n; ++i) {
            if (!own[i]) continue;
            cudaError_t e = cudaSuccess;
            if (rc == FT_OK && !st) st = gs.get(used, &e);
            if (rc == FT_OK && e != cudaSuccess) rc = ftv::cuda_fail(e);
            if (rc != FT_OK) {
                ftv::release_vote_slot(vslot[i]);
                continue;
            }
            ftv::TaskArgs a = args[i];
            a.stats = sl.host_stats_dev + i;
            ftv::VoteLaunch vl{};
            vl.max_ctas = max_ctas;
            rc = ftv::vote_task_reserved(a, st, &vl, vslot[i], sl.flags_dev + i, sl.seq);
        }
        const cudaError_t je = gs.join();
        if (rc == FT_OK && je != cudaSuccess) rc = ftv::cuda_fail(je);
        return rc;
    }
    sl.layout.build(args, tile);
    // the statistics of the batch follow the layout in the same buffer, so
    // that one upload carries the layout, its zeroed tile and done counters and the
    // initialised statistics, and no reset kernel is needed
    // (and then each request's count of voted tiles, zero)
    const size_t o_stats = ftv::BatchLayout::align(sl.layout.device_bytes());
    const size_t o_tiles = o_stats + sizeof(ft_stats) * n;
    const size_t bytes = o_tiles + sizeof(unsigned long long) * n;
    rc = grow_slot(sl, bytes, n);
    if (rc != FT_OK) return rc;
    ft_stats *dev_stats = reinterpret_cast<ft_stats *>(sl.dev + o_stats);
    // statistics of request i go to dev_stats[i]; the layout orders tasks by
    // (kind, R), so patch through its index map
    for (size_t t = 0; t < sl.layout.tasks.size(); ++t) sl.layout.tasks[t].stats = dev_stats + sl.layout.user_index[t];
    sl.layout.pack(sl.host, sl.dev, sl.gd);
    const ft_stats init = initial_stats();
    ft_stats *host_init = reinterpret_cast<ft_stats *>(sl.host + o_stats);
    for (int i = 0; i < n; ++i) host_init[i] = init;
    std::memset(sl.host + o_tiles, 0, sizeof(unsigned long long) * n);
    // the statistics go straight into the slot's pinned array, request by
    // request (without caller pointers) or by each group kernel's last CTA,
    // so no download follows the kernels; a group without tiles (only empty
    // requests) launches nothing
    for (size_t gi = 0; gi < sl.gd.size(); ++gi) {
        ftv::GroupDev &g = sl.gd[gi];
        g.warps = group_warps(sl.layout.tasks[g.t0], g.total_tiles, max_ctas);
        g.stats_base = dev_stats;
        g.stats_out = sl.host_stats_dev;
        if (any_user) {
            g.done_ctas = sl.layout.counters_dev + sl.gd.size() + gi;
        } else {
            g.tiles_done = reinterpret_cast<unsigned long long *>(sl.dev + o_tiles);
            g.flag_out = sl.flags_dev;
            g.seq = sl.seq;
        }
    }
    cudaError_t e = cudaMemcpyAsync(sl.dev, sl.host, bytes, cudaMemcpyHostToDevice, sl.stream);
    if (e != cudaSuccess) return ftv::cuda_fail(e);
    GroupStreams gs{sl};
    int launched = 0, with_tiles = 0;
    for (const ftv::GroupDev &g : sl.gd) with_tiles += g.total_tiles > 0;
    if (with_tiles > 1 && (e = gs.fork()) != cudaSuccess) return ftv::cuda_fail(e);
    for (const ftv::GroupDev &g : sl.gd) {
        if (g.total_tiles == 0) continue;
        cudaStream_t st = gs.get(launched++, &e);
        rc = e == cudaSuccess ? ftv::launch_group(g, 0, st, max_ctas) : ftv::cuda_fail(e);
        if (rc != FT_OK) {
            gs.join();
            return rc;
        }
    }
    if ((e = gs.join()) != cudaSuccess) return ftv::cuda_fail(e);
    if (any_user) {
        if ((e = cudaMemcpyAsync(sl.dev_user, sl.host_user, sizeof(ft_stats *) * n, cudaMemcpyHostToDevice,
                                 sl.stream)) != cudaSuccess)
            return ftv::cuda_fail(e);
        if ((rc = ftv::launch_stats_scatter(dev_stats, sl.dev_user, n, sl.stream)) != FT_OK) return rc;
    }
    return FT_OK;
}

// Idle time the worker spins (yielding) before it sleeps on the condition
// variable, unless the configuration says otherwise: a request that arrives
// within it is picked up without a wake-up.  A wake-up measured 50 to 70 us
// on the GPU host; at 20k requests/s (Poisson) 2 % of the gaps between
// requests exceed 200 us, and practically none exceed 2 ms.
constexpr double kSpinUs = 2000.0;

// Bound of every wait inside the resident kernel on another warp's progress
// (a tile of the largest shape takes well under a millisecond).
constexpr unsigned long long kResMaxWaitNs = 200000000ull;

// Requests of a batch stay within this factor of the batch's first request's
// bytes while another slot is free, unless the configuration says otherwise.
// At 20k requests/s with 3 streams, 93 % of the requests above the p99 latency
// had been packed into a batch with a larger one (90 % of the small ones with
// one above 100 MB), whose completion they share.  Applied on the last free
// slot too, the rule broke the 60k requests/s stream (p50 51 ms): the batches
// became too many for the slots.
constexpr unsigned long long kSizeRatio = 8;

unsigned long long size_ratio(const ft_server *s)
{
    return s->cfg.size_ratio == 0 ? kSizeRatio : s->cfg.size_ratio < 0 ? 0ull : (unsigned long long)s->cfg.size_ratio;
}

// Longest stretch the worker polls without taking the lock.
constexpr double kPollSliceUs = 50.0;

double idle_spin_us(const ft_server *s)
{
    return s->cfg.idle_spin_us == 0 ? kSpinUs : s->cfg.idle_spin_us < 0 ? 0.0 : (double)s->cfg.idle_spin_us;
}

int res_pump(ft_server *s, bool *any);
bool res_flagged(const Resident &R);
void res_stop(Resident &R);

void worker_main(ft_server *s)
{
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    double idle_since = now_us();
    for (;;) {
        // 1. completions: requests whose flags are set, and batches whose
        //    events have completed; in the shared mode also the resident
        //    kernel's, which then takes the small waiting requests
        bool any_busy = false;
        for (size_t i = 0; i < s->slots.size(); ++i) {
            if (!s->slots[i].busy) continue;
            reap_slot(s, (int)i);
            any_busy |= s->slots[i].busy;
        }
        if (s->hybrid) {
            bool moved = false;
            if (res_pump(s, &moved) > 0) any_busy = true;
            if (moved) idle_since = now_us();
        }
        if (s->stop && !any_busy) break;
        int free_slot = -1;
        for (size_t i = 0; i < s->slots.size(); ++i)
            if (!s->slots[i].busy) { free_slot = (int)i; break; }
        // 2. nothing to launch: spin while batches are in flight or shortly
        //    after the last activity, else sleep until a request or stop
        if (s->stop || s->paused || s->pending.empty() || free_slot < 0) {
            if (any_busy || now_us() - idle_since < idle_spin_us(s)) {
                // wait for a change without holding the lock, so that clients
                // calling ft_submit / ft_poll meanwhile never queue behind
                // the worker: a new request, pause or stop (the state
                // version), a request's flag, or a batch's event completing
                // (only this thread changes the slots)
                const unsigned long long ver = s->version.load(std::memory_order_acquire);
                const double t_end = now_us() + kPollSliceUs;
                lk.unlock();
                for (bool changed = false; !changed && now_us() < t_end;) {
                    changed = s->version.load(std::memory_order_acquire) != ver;
                    for (size_t k = 0; k < s->slots.size() && !changed; ++k)
                        if (s->slots[k].busy) changed = slot_progress(s->slots[k]);
                    if (!changed && s->hybrid) changed = res_flagged(s->res);
                    if (!changed && !any_busy) std::this_thread::yield();
                }
                lk.lock();
            } else {
                s->cv_work.wait(lk);
                idle_since = now_us();
            }
            continue;
        }
        // 3. take up to max_slots waiting requests (FIFO) into this slot
        Slot &sl = s->slots[free_slot];
        std::vector<ftv::TaskArgs> args;
        sl.tickets.clear();
        bool any_user = false;
        unsigned long long batch_bytes = 0, first_bytes = 0;
        std::vector<unsigned long long> req_bytes;
        // the size rule holds only while another slot is free for the requests
        // it leaves waiting; on the last free slot everything waiting is packed
        int free_slots = 0;
        for (const Slot &o : s->slots) free_slots += !o.busy;
        const unsigned long long ratio = free_slots >= 2 ? size_ratio(s) : 0;
        // the waiting requests are spread evenly over the free slots: while
        // as many slots are free as requests wait, each request gets a batch
        // of its own (nothing to gain from packing with a slot to spare);
        // packing starts once the requests outnumber the free slots.  At 20k
        // requests/s on 4 streams, p99 over three replays: 168-171 us packing
        // everything waiting, 164-166 us spread.
        const size_t kmax =
            std::min((size_t)s->cfg.max_slots, (s->pending.size() + (size_t)free_slots - 1) / (size_t)free_slots);
        while (!s->pending.empty() && args.size() < kmax) {
            const unsigned long long tk = s->pending.front();
            auto it = s->reqs.find(tk);
            if (it == s->reqs.end()) {
                s->pending.pop_front();
                continue;
            }
            const unsigned long long rb = it->second.bytes;
            if (!args.empty() && s->cfg.max_batch_bytes && batch_bytes + rb > s->cfg.max_batch_bytes) break;
            // a request far smaller or larger than the batch's first waits for
            // the next batch: a small one would otherwise complete only with
            // the large one it was packed with
            // (empty requests cost nothing and go with any batch)
            if (ratio && rb && first_bytes && (rb > ratio * first_bytes || ratio * rb < first_bytes)) break;
            if (!first_bytes) first_bytes = rb;
            s->pending.pop_front();
            s->queue_us += now_us() - it->second.submit_us;
            batch_bytes += it->second.bytes;
            args.push_back(it->second.args);
            req_bytes.push_back(rb);
            sl.tickets.push_back(tk);
            any_user |= it->second.user_stats != nullptr;
        }
        if (args.empty()) continue;
        if (args.size() > 1) {
            // smallest first: the batch's tiles are voted in request order
            // (within each element type / R group), so its small requests
            // complete, each on its own, before its large ones
            std::vector<int> ord(args.size());
            for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
            std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return req_bytes[x] < req_bytes[y]; });
            std::vector<ftv::TaskArgs> a2(args.size());
            std::vector<unsigned long long> t2(args.size());
            for (size_t i = 0; i < ord.size(); ++i) {
                a2[i] = args[ord[i]];
                t2[i] = sl.tickets[ord[i]];
            }
            args.swap(a2);
            sl.tickets.swap(t2);
        }
        sl.busy = true;
        s->batches += 1;
        s->batched_requests += args.size();
        s->busy_now += 1;
        s->busy_max = std::max(s->busy_max, s->busy_now);
        std::vector<ft_stats *> users(args.size());
        for (size_t i = 0; i < args.size(); ++i) users[i] = s->reqs[sl.tickets[i]].user_stats;
        sl.seq = ++s->batch_seq;
        sl.req_done.assign(args.size(), 0);
        sl.ndone = 0;
        sl.per_req = false;
        sl.ended = false;
        lk.unlock();
        sl.launched_at = now_us();
        sl.last_check = sl.launched_at;
        int rc = FT_OK;
        if (any_user) {
            rc = grow_slot(sl, 0, (int)args.size());
            if (rc == FT_OK) std::memcpy(sl.host_user, users.data(), sizeof(ft_stats *) * users.size());
        }
        if (rc == FT_OK) rc = launch_slot(s, free_slot, args, any_user);
        sl.status = rc;
        sl.per_req = rc == FT_OK && !any_user;
        cudaError_t e = cudaEventRecord(sl.done, sl.stream);
        sl.launch_done_at = now_us();
        const double launched = sl.launch_done_at - sl.launched_at;
        if (e != cudaSuccess) {
            // no completion event: finish the batch here
            cudaStreamSynchronize(sl.stream);
            sl.status = ftv::cuda_fail(e);
            lk.lock();
            s->launch_host_us += launched;
            complete_slot(s, free_slot, now_us());
        } else {
            lk.lock();
            s->launch_host_us += launched;
        }
        idle_since = now_us();
    }
    if (s->resident) {
        lk.unlock();
        res_stop(s->res);
    }
}

// ---------------------------------------------------------------------------
// Resident mode
// ---------------------------------------------------------------------------

// Tile of a resident request: about one tile per voting warp (up to 64
// blocks), so a small request is spread over as many warps as it has blocks
// and a large one is claimed once per warp.
void res_tiles(const ft_server *s, const ftv::TaskArgs &a, unsigned long long *ntiles, int *tile_blocks)
{
    const unsigned long long nblk = a.nfull + (a.tail_bytes ? 1ull : 0ull);
    const unsigned long long v = (unsigned long long)std::max(1, s->res.voting_warps);
    // about one tile per voting warp (each claim and count is a round trip
    // to a shared counter), at most 64 blocks
    const unsigned long long tb = std::min(64ull, std::max(1ull, (nblk + v - 1ull) / v));
    *tile_blocks = (int)tb;
    *ntiles = nblk ? (nblk + (unsigned long long)tb - 1ull) / (unsigned long long)tb : 1ull;
}

// Request of slot j is done with `status` (lock held).
void res_complete(ft_server *s, int j, double t, int status)
{
    Resident &R = s->res;
    auto it = s->reqs.find(R.slot_ticket[j]);
    if (it != s->reqs.end()) {
        Request &r = it->second;
        r.result = status == FT_OK ? R.stats_out[j] : initial_stats();
        r.status = status;
        r.done = true;
        r.done_us = t;
    }
    s->completed += 1;
    s->batch_span_us += t - R.slot_sent[j];
    s->busy_now -= 1;
    R.slot_gen[j] = 0;
    s->cv_done.notify_all();
}

// Completions seen in the flags (lock held); returns the slots still busy.
int res_reap(ft_server *s, double t, bool *any)
{
    Resident &R = s->res;
    int busy = 0;
    for (int j = 0; j < ftv::kResSlots; ++j) {
        if (!R.slot_gen[j]) continue;
        if (__atomic_load_n(&R.flags[j], __ATOMIC_ACQUIRE) == R.slot_gen[j]) {
            res_complete(s, j, t, FT_OK);
            *any = true;
        } else {
            ++busy;
        }
    }
    return busy;
}

// Hands request tk to free slot j (lock held).
void res_send_request(ft_server *s, int j, unsigned long long tk, Request &r)
{
    Resident &R = s->res;
    const double t0 = now_us();
    ftv::ResMail &m = R.mail[j];
    m.args = r.args;
    m.args.stats = R.g.stats + j;
    m.user = r.user_stats;
    res_tiles(s, r.args, &m.ntiles, &m.tile_blocks);
    // small: fewer blocks than voting warps
    m.urgent = r.args.nfull + (r.args.tail_bytes ? 1ull : 0ull) < (unsigned long long)R.voting_warps;
    m.gen = ++R.gen;
    m.pad_ = 0;
    R.slot_gen[j] = m.gen;
    R.slot_ticket[j] = tk;
    // the mailbox is written before its generation is published
    __atomic_store_n(&R.mail_gen[j], m.gen, __ATOMIC_RELEASE);
    const double t1 = now_us();
    R.slot_sent[j] = t1;
    r.launch_us = t0;
    r.launched_us = t1;
    s->queue_us += t0 - r.submit_us;
    s->launch_host_us += t1 - t0;
    s->batches += 1;
    s->batched_requests += 1;
    s->busy_now += 1;
    s->busy_max = std::max(s->busy_max, s->busy_now);
}

// Hands the oldest waiting request to free slot j (lock held).
bool res_send(ft_server *s, int j)
{
    while (!s->pending.empty()) {
        const unsigned long long tk = s->pending.front();
        s->pending.pop_front();
        auto it = s->reqs.find(tk);
        if (it == s->reqs.end()) continue;
        res_send_request(s, j, tk, it->second);
        return true;
    }
    return false;
}

// The kernel has left (or failed): with an error every request on the
// device fails, and so do the waiting ones (lock held).
void res_fail_all(ft_server *s, int status, double t)
{
    Resident &R = s->res;
    for (int j = 0; j < ftv::kResSlots; ++j)
        if (R.slot_gen[j]) res_complete(s, j, t, status);
    while (!s->pending.empty()) {
        auto it = s->reqs.find(s->pending.front());
        s->pending.pop_front();
        if (it == s->reqs.end()) continue;
        it->second.result = initial_stats();
        it->second.status = status;
        it->second.done = true;
        it->second.done_us = t;
    }
    s->cv_done.notify_all();
}

// Whether the resident kernel has left; notes a failure (lock held or not:
// only the worker touches these fields).
bool res_left(Resident &R)
{
    const cudaError_t q = cudaEventQuery(R.done);
    if (q == cudaErrorNotReady) return false;
    R.running = false;
    if (q != cudaSuccess) R.failed = ftv::cuda_fail(q);
    else if (__atomic_load_n(R.error, __ATOMIC_ACQUIRE) != 0u) R.failed = FT_ECUDA;
    return true;
}

// The shared mode (ft_server_config.resident = 2), from the batch worker
// (lock held): completions of the resident kernel, and every waiting request
// with fewer blocks than the kernel's voting warps handed to it while it has
// free slots; the kernel is launched when its slots are busy and it is not
// running.  Returns its busy slots.  After a failure of the kernel its
// requests fail and every later request takes the batches.
int res_pump(ft_server *s, bool *any)
{
    Resident &R = s->res;
    const double t = now_us();
    int busy = res_reap(s, t, any);
    if (R.running && t - R.last_query >= kEventCheckUs) {
        R.last_query = t;
        if (res_left(R)) busy = res_reap(s, t, any);
    }
    if (R.failed != FT_OK) {
        for (int j = 0; j < ftv::kResSlots; ++j)
            if (R.slot_gen[j]) res_complete(s, j, t, R.failed);
        s->hybrid = false;
        return 0;
    }
    if (!s->stop && !s->paused) {
        int j = 0;
        for (auto it = s->pending.begin(); it != s->pending.end() && busy < ftv::kResSlots;) {
            auto rq = s->reqs.find(*it);
            if (rq == s->reqs.end()) {
                it = s->pending.erase(it);
                continue;
            }
            const ftv::TaskArgs &a = rq->second.args;
            if (a.nfull + (a.tail_bytes ? 1ull : 0ull) >= (unsigned long long)R.voting_warps) {
                ++it;
                continue;
            }
            while (R.slot_gen[j]) ++j;
            res_send_request(s, j, *it, rq->second);
            it = s->pending.erase(it);
            ++busy;
            *any = true;
        }
    }
    if (busy && !R.running) {
        R.g.epoch += 1;
        int ctas = 0;
        int rc = ftv::resident_launch(R.g, R.stream, R.max_ctas, &ctas);
        cudaError_t e = cudaSuccess;
        if (rc == FT_OK && (e = cudaEventRecord(R.done, R.stream)) != cudaSuccess) rc = ftv::cuda_fail(e);
        if (rc != FT_OK) {
            R.failed = rc;
            return res_pump(s, any);
        }
        R.running = true;
        R.launches += 1;
        R.last_query = now_us();
    }
    return busy;
}

// Whether the resident kernel has completed a request (no lock: only the
// worker changes the slots).
bool res_flagged(const Resident &R)
{
    for (int j = 0; j < ftv::kResSlots; ++j)
        if (R.slot_gen[j] && __atomic_load_n(&R.flags[j], __ATOMIC_ACQUIRE) == R.slot_gen[j]) return true;
    return false;
}

// Tells the resident kernel to leave and waits for it (its waits are bounded).
void res_stop(Resident &R)
{
    __atomic_store_n(R.quit, 1u, __ATOMIC_RELEASE);
    if (R.running) cudaEventSynchronize(R.done);
    R.running = false;
}

void res_worker(ft_server *s)
{
    cudaSetDevice(s->device);
    Resident &R = s->res;
    std::unique_lock<std::mutex> lk(s->mu);
    double idle_since = now_us();
    for (;;) {
        double t = now_us();
        bool any = false;
        int busy = res_reap(s, t, &any);
        // the kernel: has it left?  (queried at most every kEventCheckUs,
        // and not while a request waits to be handed over)
        if (R.running && t - R.last_query >= kEventCheckUs && (busy > 0 || s->pending.empty())) {
            R.last_query = t;
            if (res_left(R)) busy = res_reap(s, t, &any);   // its last flags
        }
        if (R.failed != FT_OK) {
            res_fail_all(s, R.failed, t);
            busy = 0;
        }
        if (s->stop && busy == 0) break;
        // waiting requests to free slots
        if (!s->stop && !s->paused && R.failed == FT_OK) {
            for (int j = 0; j < ftv::kResSlots && !s->pending.empty(); ++j)
                if (!R.slot_gen[j] && res_send(s, j)) {
                    ++busy;
                    any = true;
                }
        }
        // the kernel runs while any slot is busy (it leaves by itself once
        // idle; a request handed over as it left finds it gone here)
        if (busy && !R.running && R.failed == FT_OK) {
            R.g.epoch += 1;
            int ctas = 0;
            int rc = ftv::resident_launch(R.g, R.stream, R.max_ctas, &ctas);
            cudaError_t e = cudaSuccess;
            if (rc == FT_OK && (e = cudaEventRecord(R.done, R.stream)) != cudaSuccess) rc = ftv::cuda_fail(e);
            if (rc != FT_OK) {
                R.failed = rc;
                continue;
            }
            R.running = true;
            R.launches += 1;
            R.last_query = now_us();
        }
        if (any || busy) idle_since = now_us();
        // wait: poll while requests are on the device or shortly after the
        // last activity, without holding the lock; else sleep
        if (busy || now_us() - idle_since < idle_spin_us(s)) {
            const unsigned long long ver = s->version.load(std::memory_order_acquire);
            const double t_end = now_us() + kPollSliceUs;
            lk.unlock();
            for (bool changed = false; !changed && now_us() < t_end;) {
                changed = s->version.load(std::memory_order_acquire) != ver;
                for (int j = 0; j < ftv::kResSlots && !changed; ++j)
                    changed = R.slot_gen[j] && __atomic_load_n(&R.flags[j], __ATOMIC_ACQUIRE) == R.slot_gen[j];
                if (!changed && !busy) std::this_thread::yield();
            }
            lk.lock();
        } else {
            s->cv_work.wait(lk);
            idle_since = now_us();
        }
    }
    lk.unlock();
    res_stop(R);
}

// Device and host-mapped memory of the resident mode, the kernel loaded.
int res_init(ft_server *s)
{
    Resident &R = s->res;
    using ftv::kResSlots;
    cudaError_t e;
    int rc = ftv::resident_preload(R.max_ctas, &R.voting_warps);
    if (rc != FT_OK) return rc;
    if ((e = cudaStreamCreateWithFlags(&R.stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&R.done, cudaEventDisableTiming)) != cudaSuccess)
        return ftv::cuda_fail(e);
    // device block: slots | next | meta | done | admitted | fin | beat, progress | active, urgent, stop | stats
    const size_t o_slots = 0;
    const size_t o_next = o_slots + sizeof(ftv::ResSlot) * kResSlots;
    const size_t o_meta = o_next + 8 * kResSlots;
    const size_t o_done = o_meta + 8 * kResSlots;
    const size_t o_adm = o_done + 8 * kResSlots;
    const size_t o_fin = o_adm + 8 * kResSlots;
    const size_t o_beat = o_fin + 8 * kResSlots;
    const size_t o_act = o_beat + 16;
    const size_t o_stats = (o_act + 16 + 255) & ~size_t(255);
    const size_t dev_bytes = o_stats + sizeof(ft_stats) * kResSlots;
    // host-mapped block: mailboxes | mail_gen | flags | quit, error | stats copies
    const size_t h_mail = 0;
    const size_t h_gen = h_mail + sizeof(ftv::ResMail) * kResSlots;
    const size_t h_flags = h_gen + 8 * kResSlots;
    const size_t h_ctl = h_flags + 8 * kResSlots;
    const size_t h_stats = (h_ctl + 8 + 255) & ~size_t(255);
    const size_t host_bytes = h_stats + sizeof(ft_stats) * kResSlots;
    if ((e = cudaMalloc(&R.dev, dev_bytes)) != cudaSuccess) return ftv::cuda_fail(e);
    if ((e = cudaHostAlloc(reinterpret_cast<void **>(&R.host), host_bytes, cudaHostAllocMapped)) != cudaSuccess)
        return ftv::cuda_fail(e);
    std::memset(R.host, 0, host_bytes);
    uint8_t *hd = nullptr;
    if ((e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&hd), R.host, 0)) != cudaSuccess)
        return ftv::cuda_fail(e);
    // the device block at its initial values: zero counters, initial statistics
    std::vector<uint8_t> init(dev_bytes, 0);
    const ft_stats st0 = initial_stats();
    for (int j = 0; j < kResSlots; ++j) std::memcpy(init.data() + o_stats + sizeof(ft_stats) * j, &st0, sizeof(st0));
    if ((e = cudaMemcpy(R.dev, init.data(), dev_bytes, cudaMemcpyHostToDevice)) != cudaSuccess)
        return ftv::cuda_fail(e);
    R.mail = reinterpret_cast<ftv::ResMail *>(R.host + h_mail);
    R.mail_gen = reinterpret_cast<unsigned long long *>(R.host + h_gen);
    R.flags = reinterpret_cast<unsigned long long *>(R.host + h_flags);
    R.quit = reinterpret_cast<unsigned int *>(R.host + h_ctl);
    R.error = R.quit + 1;
    R.stats_out = reinterpret_cast<ft_stats *>(R.host + h_stats);
    ftv::ResDev &g = R.g;
    g.mail = reinterpret_cast<const ftv::ResMail *>(hd + h_mail);
    g.mail_gen = reinterpret_cast<const unsigned long long *>(hd + h_gen);
    g.flags = reinterpret_cast<unsigned long long *>(hd + h_flags);
    g.quit = reinterpret_cast<const unsigned int *>(hd + h_ctl);
    g.error = reinterpret_cast<unsigned int *>(hd + h_ctl) + 1;
    g.stats_out = reinterpret_cast<ft_stats *>(hd + h_stats);
    g.slots = reinterpret_cast<ftv::ResSlot *>(R.dev + o_slots);
    g.next = reinterpret_cast<unsigned long long *>(R.dev + o_next);
    g.meta = reinterpret_cast<unsigned long long *>(R.dev + o_meta);
    g.done = reinterpret_cast<unsigned long long *>(R.dev + o_done);
    g.admitted = reinterpret_cast<unsigned long long *>(R.dev + o_adm);
    g.fin = reinterpret_cast<unsigned long long *>(R.dev + o_fin);
    g.beat = reinterpret_cast<unsigned long long *>(R.dev + o_beat);
    g.progress = g.beat + 1;
    g.active = reinterpret_cast<unsigned int *>(R.dev + o_act);
    g.urgent = g.active + 1;
    g.stop = g.active + 2;
    g.stats = reinterpret_cast<ft_stats *>(R.dev + o_stats);
    const double idle_us = idle_spin_us(s) > 0.0 ? idle_spin_us(s) : kSpinUs;
    g.idle_ns = (unsigned long long)(idle_us * 1e3);
    g.max_wait_ns = kResMaxWaitNs;
    g.epoch = 0;
    return FT_OK;
}

void res_free(Resident &R)
{
    if (R.running && R.quit) {
        __atomic_store_n(R.quit, 1u, __ATOMIC_RELEASE);
        cudaEventSynchronize(R.done);
    }
    if (R.stream) cudaStreamSynchronize(R.stream);
    if (R.done) cudaEventDestroy(R.done);
    if (R.stream) cudaStreamDestroy(R.stream);
    if (R.dev) cudaFree(R.dev);
    if (R.host) cudaFreeHost(R.host);
}

void free_server(ft_server *s)
{
    if (s->resident) res_free(s->res);
    for (auto &sl : s->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.dev) cudaFree(sl.dev);
        if (sl.host) cudaFreeHost(sl.host);
        if (sl.host_stats) cudaFreeHost(sl.host_stats);
        if (sl.flags) cudaFreeHost(sl.flags);
        if (sl.dev_user) cudaFree(sl.dev_user);
        if (sl.host_user) cudaFreeHost(sl.host_user);
        if (sl.small_area) cudaFree(sl.small_area);
        for (int a = 0; a < kAuxStreams; ++a) {
            if (sl.aux[a]) {
                cudaStreamSynchronize(sl.aux[a]);
                cudaStreamDestroy(sl.aux[a]);
            }
            if (sl.joined[a]) cudaEventDestroy(sl.joined[a]);
        }
        if (sl.forked) cudaEventDestroy(sl.forked);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    delete s;
}

}  // namespace

extern "C" {

int ft_server_create(ft_server **out, const ft_server_config *cfg)
{
    if (!out || !cfg) return FT_EINVAL;
    *out = nullptr;
    if (cfg->mem_budget_bytes == 0 || cfg->max_slots < 1 || cfg->max_slots > 65536 || cfg->streams < 1 ||
        cfg->streams > 8 || cfg->tile_blocks < 0 || cfg->tile_blocks > 64 || cfg->max_inflight < 0 ||
        cfg->reserved_sms < -1 || cfg->idle_spin_us < -1 || cfg->size_ratio < -1 || cfg->size_ratio == 1 ||
        cfg->resident < 0 || cfg->resident > 2)
        return FT_EINVAL;
    ft_server *s = new (std::nothrow) ft_server();
    if (!s) return FT_ENOMEM;
    s->cfg = *cfg;
    s->auto_tile = cfg->tile_blocks == 0;
    if (s->cfg.tile_blocks == 0) s->cfg.tile_blocks = 8;
    if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 65536;
    cudaError_t e = cudaGetDevice(&s->device);
    if (e != cudaSuccess) {
        delete s;
        return ftv::cuda_fail(e);
    }
    if (cfg->resident == 1) {
        s->resident = true;
        int rc = res_init(s);
        if (rc != FT_OK) {
            free_server(s);
            return rc == FT_ECUDA && ftv::g_last_cuda == cudaErrorMemoryAllocation ? FT_ENOMEM : rc;
        }
        s->worker = std::thread(res_worker, s);
        *out = s;
        return FT_OK;
    }
    s->slots.resize(cfg->streams);
    int rc = FT_OK;
    // size each slot for a batch that fills the whole budget
    const unsigned long long tiles = cfg->mem_budget_bytes / (2ull * 4096ull * s->cfg.tile_blocks) + cfg->max_slots;
    const size_t guess = sizeof(ftv::TaskArgs) * cfg->max_slots + 8ull * cfg->max_slots + 4ull * tiles + 4096 +
                         sizeof(ft_stats) * (size_t)std::min(cfg->max_slots, 4096);
    for (auto &sl : s->slots) {
        if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&sl.forked, cudaEventDisableTiming)) != cudaSuccess) {
            rc = ftv::cuda_fail(e);
            break;
        }
        for (int a = 0; a < kAuxStreams && e == cudaSuccess; ++a)
            if ((e = cudaStreamCreateWithFlags(&sl.aux[a], cudaStreamNonBlocking)) == cudaSuccess)
                e = cudaEventCreateWithFlags(&sl.joined[a], cudaEventDisableTiming);
        if (e != cudaSuccess) {
            rc = ftv::cuda_fail(e);
            break;
        }
        if ((rc = grow_slot(sl, guess, std::min(cfg->max_slots, 4096))) != FT_OK) break;
        if ((e = cudaMalloc(&sl.small_area, kSmallAreaBytes)) != cudaSuccess) {
            rc = ftv::cuda_fail(e);
            break;
        }
        sl.small_cnt = reinterpret_cast<unsigned long long *>(sl.small_area);
        sl.small_tiles = sl.small_cnt + 2 * ftv::kSmallTasks;
        sl.small_stats = reinterpret_cast<ft_stats *>(sl.small_area + kSmallCntBytes);
    }
    // every kernel a request may launch is loaded now, not at the request's launch
    if (rc == FT_OK && (rc = ftv::preload_vote_kernels()) == FT_OK) rc = ftv::preload_group_kernels();
    if (rc == FT_OK && cfg->resident == 2) {
        // the resident kernel on the SMs the batches leave free
        s->resident = s->hybrid = true;
        const int reserve = cfg->reserved_sms > 0 ? cfg->reserved_sms : kReservedSms;
        s->res.max_ctas = reserve;
        rc = res_init(s);
    }
    if (rc != FT_OK) {
        free_server(s);
        return rc == FT_ECUDA && ftv::g_last_cuda == cudaErrorMemoryAllocation ? FT_ENOMEM : rc;
    }
    s->worker = std::thread(worker_main, s);
    *out = s;
    return FT_OK;
}

}  // extern "C"

namespace {

// Validates one request and fills everything but its ticket (no lock held).
int prepare_request(const ft_server *s, const ft_vote_desc *desc, Request &r)
{
    if (!desc) return FT_EINVAL;
    // the server supplies the statistics buffer when the caller gives none
    ft_vote_desc d = *desc;
    ft_stats dummy;
    const bool user = d.stats != nullptr;
    if (!user) d.stats = &dummy;
    const int rc = ftv::validate_desc(&d);
    if (rc != FT_OK) return rc;
    const unsigned long long bytes = (unsigned long long)(d.R + 1) * d.n * ftv::dtype_size(d.dtype);
    if (bytes > s->cfg.mem_budget_bytes) return FT_EINVAL;   // can never be admitted
    r.args = ftv::make_task_args(&d);
    r.user_stats = user ? desc->stats : nullptr;
    r.bytes = bytes;
    r.submit_us = now_us();
    return FT_OK;
}

// Admits a prepared request (lock held): FT_OK with its ticket, or FT_EAGAIN.
int admit_locked(ft_server *s, const Request &r, uint64_t *ticket)
{
    if (s->inflight_bytes + r.bytes > s->cfg.mem_budget_bytes || s->inflight >= s->cfg.max_inflight) return FT_EAGAIN;
    const unsigned long long t = s->next_ticket++;
    s->reqs.emplace(t, r);
    s->pending.push_back(t);
    s->version.fetch_add(1, std::memory_order_release);
    s->inflight_bytes += r.bytes;
    s->inflight += 1;
    *ticket = t;
    return FT_OK;
}

// Waits (lock held) up to timeout_us (< 0: no limit, 0: not at all) for a
// ticket: FT_OK when it is done, FT_ETIMEDOUT, or FT_ENOTFOUND.
int wait_done_locked(ft_server *s, std::unique_lock<std::mutex> &lk, uint64_t ticket, int64_t timeout_us)
{
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return FT_ENOTFOUND;
    if (it->second.done) return FT_OK;
    auto ready = [&] {
        auto j = s->reqs.find(ticket);
        return j == s->reqs.end() || j->second.done;
    };
    if (timeout_us < 0) {
        s->cv_done.wait(lk, ready);
    } else if (timeout_us > 0) {
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    }
    it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return FT_ENOTFOUND;
    return it->second.done ? FT_OK : FT_ETIMEDOUT;
}

// Retires a done request (lock held), filling *res when it is not NULL.
void retire_locked(ft_server *s, std::unordered_map<unsigned long long, Request>::iterator it, ft_result *res)
{
    Request &r = it->second;
    if (res) {
        res->status = r.status;
        res->R = r.args.R;
        res->n = r.args.n;
        res->stats = r.result;
        res->submit_us = r.submit_us;
        res->done_us = r.done_us;
        res->launch_us = r.launch_us;
        res->launched_us = r.launched_us;
    }
    s->inflight_bytes -= r.bytes;
    s->inflight -= 1;
    s->reqs.erase(it);
}

}  // namespace

extern "C" {

int ft_submit(ft_server *s, const ft_vote_desc *desc, uint64_t *ticket)
{
    if (!s || !desc || !ticket) return FT_EINVAL;
    Request r;
    int rc = prepare_request(s, desc, r);
    if (rc != FT_OK) return rc;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return FT_EINVAL;
    if ((rc = admit_locked(s, r, ticket)) == FT_OK) s->cv_work.notify_one();
    return rc;
}

int ft_submit_many(ft_server *s, const ft_vote_desc *const *descs, int32_t n, uint64_t *tickets, int32_t *accepted)
{
    if (!s || !accepted || n < 0 || (n > 0 && (!descs || !tickets))) return FT_EINVAL;
    *accepted = 0;
    std::vector<Request> rs(n);
    int valid = 0, rc_bad = FT_OK;
    for (; valid < n; ++valid)
        if ((rc_bad = prepare_request(s, descs[valid], rs[valid])) != FT_OK) break;
    int k = 0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return FT_EINVAL;
        for (; k < valid; ++k)
            if (admit_locked(s, rs[k], &tickets[k]) != FT_OK) break;
        if (k > 0) s->cv_work.notify_one();
    }
    *accepted = k;
    return (k == valid && valid < n) ? rc_bad : FT_OK;
}

int ft_poll(ft_server *s, uint64_t ticket, int64_t timeout_us, ft_result *res)
{
    if (!s) return FT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    const int rc = wait_done_locked(s, lk, ticket, timeout_us);
    if (rc != FT_OK) return rc;
    retire_locked(s, s->reqs.find(ticket), res);
    return FT_OK;
}

int ft_poll_many(ft_server *s, const uint64_t *tickets, int32_t n, int64_t timeout_us, ft_result *results,
                 int32_t *ndone)
{
    if (!s || !ndone || n < 0 || (n > 0 && !tickets)) return FT_EINVAL;
    *ndone = 0;
    if (n == 0) return FT_OK;
    std::unique_lock<std::mutex> lk(s->mu);
    int rc = wait_done_locked(s, lk, tickets[0], timeout_us);
    if (rc != FT_OK) return rc;
    int k = 0;
    for (; k < n; ++k) {
        auto it = s->reqs.find(tickets[k]);
        if (it == s->reqs.end()) {
            rc = FT_ENOTFOUND;
            break;
        }
        if (!it->second.done) break;
        retire_locked(s, it, results ? &results[k] : nullptr);
    }
    *ndone = k;
    return rc;
}

int ft_server_pause(ft_server *s, int32_t paused)
{
    if (!s) return FT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    s->paused = paused != 0;
    s->version.fetch_add(1, std::memory_order_release);
    s->cv_work.notify_all();
    return FT_OK;
}

int ft_server_destroy(ft_server *s)
{
    if (!s) return FT_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->pending.clear();
        s->version.fetch_add(1, std::memory_order_release);
        s->cv_work.notify_all();
    }
    if (s->worker.joinable()) s->worker.join();
    free_server(s);
    return FT_OK;
}

int ft_server_info(ft_server *s, ft_server_stats *out)
{
    if (!s || !out) return FT_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    out->batches = s->batches;
    out->requests = s->batched_requests;
    out->completed = s->completed;
    out->max_batches_in_flight = s->busy_max;
    out->inflight_requests = s->inflight;
    out->inflight_bytes = s->inflight_bytes;
    out->launch_host_us = s->launch_host_us;
    out->batch_span_us = s->batch_span_us;
    out->queue_us = s->queue_us;
    return FT_OK;
}

double ft_clock_us(void) { return now_us(); }

}  // extern "C"
