// resident.h -- the server's resident voter: one persistent kernel that stays
// on the GPU while vote requests arrive, takes each request from a
// host-mapped mailbox and votes it in tiles, the request with the fewest
// tiles left first, with no kernel launch per request.
#pragma once

#include <cstdint>

#include "common.cuh"
#include "runtime.h"

namespace ftv {

// Requests on the device at once: one mailbox and one device slot each (one
// per lane of the warp that scans them).
constexpr int kResSlots = 32;
// next[j] and meta[j] hold (generation mod 2^24) << 40 | a tile count: tiles
// claimed so far and tiles of the request.  A claim is valid only if the
// generation it returns is the one the claiming warp scanned.
constexpr int kResGenShift = 40;
constexpr unsigned long long kResTileMask = (1ull << kResGenShift) - 1ull;

// A request as the host hands it over (host-mapped memory, one per slot).
// The host writes it, then publishes gen in mail_gen[slot].
struct ResMail {
    TaskArgs args;             // args.stats = the slot's device statistics
    ft_stats *user;            // the caller's device statistics, or null
    unsigned long long ntiles; // >= 1 (a request of no elements is one tile of nothing)
    unsigned long long gen;    // the request's generation, > 0, unique per server
    int32_t tile_blocks;       // 4 KiB blocks per tile
    int32_t urgent;            // 1 = small: warps voting other requests' tiles stop between blocks for it
    unsigned long long pad_;   // to a multiple of 16 bytes (the kernel copies it 16 bytes at a time)
};

// The same on the device, copied in by the admitting warp.
struct ResSlot {
    TaskArgs args;
    ft_stats *user;
    unsigned long long ntiles;
    unsigned long long gen;
    int32_t tile_blocks;
    int32_t urgent;
    unsigned long long pad_;
};
static_assert(sizeof(ResMail) == sizeof(ResSlot) && sizeof(ResMail) % 16 == 0, "mailbox layout");

// Error codes the kernel leaves in *error (host-mapped).
constexpr unsigned int kResErrNoBeat = 1;      // a voting warp saw the admitting warp stop beating
constexpr unsigned int kResErrNoProgress = 2;  // requests on the device, none completed for max_wait_ns

struct ResDev {
    const ResMail *mail;                 // host-mapped: kResSlots mailboxes
    const unsigned long long *mail_gen;  // host-mapped: generation published per slot (0 = none yet)
    const unsigned int *quit;            // host-mapped: nonzero = leave now
    unsigned int *error;                 // host-mapped: a kResErr* code, 0 = none
    ResSlot *slots;                      // device: the admitted requests
    unsigned long long *next;            // device: claim counters (generation | tiles claimed)
    unsigned long long *meta;            // device: generation | tiles of the request
    unsigned long long *done;            // device: tiles voted (0 between requests)
    unsigned long long *admitted;        // device: generation last copied in, per slot
    unsigned long long *fin;             // device: generation last completed, per slot
    unsigned long long *beat;            // device: the admitting warp's loop count
    unsigned long long *progress;        // device: requests completed since the server started
    unsigned int *active;                // device: bit j = slot j may have unclaimed tiles
    unsigned int *urgent;                // device: the same for the small requests
    unsigned int *stop;                  // device: epoch of the launch whose admitting warp has left
    ft_stats *stats;                     // device: per-slot statistics, initial values between requests
    ft_stats *stats_out;                 // host-mapped: each request's statistics, written before its flag
    unsigned long long *flags;           // host-mapped: the request's generation once it is done
    unsigned long long idle_ns;          // the admitting warp leaves after this long with nothing to do
    unsigned long long max_wait_ns;      // bound of every wait on another warp
    unsigned int epoch;                  // this launch
    unsigned int pad_;
};

// Warps per CTA of the resident kernel (one CTA per SM: the CRC tables take
// the shared memory).  Warp 0 of CTA 0 admits requests; every other warp votes.
constexpr int kResWarps = 16;

// Launches the resident kernel on s: one CTA per SM, at most max_ctas of
// them (0 = every SM; grid returned in *ctas).  It returns once nothing has
// arrived for idle_ns and every admitted request is done, or at once when
// *quit is set.
int resident_launch(const ResDev &g, cudaStream_t s, int max_ctas, int *ctas);
// Loads the kernel and sets its shared-memory size (at server creation, so
// that no request pays the lazy module load); *voting_warps = the warps that
// vote in one launch of at most max_ctas CTAs.
int resident_preload(int max_ctas, int *voting_warps);

}  // namespace ftv
