// registry.cpp -- value types of registered buffers, and task duplication.
//
// In the paper's API an application registers each memory area with its value
// type and access mode (dls_register_data(ptr, size, DLS_VT_FLOAT, "w"),
// Sec. IV.E); the value type decides how the voter compares results (bit-wise
// for integers, within a delta for floats; Sec. IV.D).  ft_register_data keeps
// the same information for device buffers, and ft_vote_registered votes into a
// registered output area with its registered type and tolerances.
//
// ft_dmr_run is the task duplication of Sec. IV.D: it runs a caller-supplied
// task once per replica buffer (the task may pick a different kernel or
// processing unit per replica, as the HetDMR mode does), then votes.
#include <cstring>
#include <iterator>
#include <map>
#include <mutex>

#include <cuda_runtime.h>

#include "ftvote.h"
#include "runtime.h"

namespace {

struct Area {
    uint64_t bytes;
    int32_t dtype;
    double abs_tol, rel_tol;
};

std::mutex g_reg_mu;
std::map<uintptr_t, Area> g_reg;   // keyed by start address

// The registered area containing p, or end().
std::map<uintptr_t, Area>::const_iterator find_area(const void *p)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    auto it = g_reg.upper_bound(a);
    if (it == g_reg.begin()) return g_reg.end();
    --it;
    return a < it->first + it->second.bytes ? it : g_reg.end();
}

}  // namespace

extern "C" {

int ft_register_data(const void *ptr, uint64_t bytes, int32_t dtype, double abs_tol, double rel_tol)
{
    const size_t sz = ftv::dtype_size(dtype);
    if (!ptr || bytes == 0 || sz == 0 || bytes % sz) return FT_EINVAL;
    if (dtype == FT_F32 || dtype == FT_F64) {
        if (!(abs_tol >= 0.0) || !(rel_tol >= 0.0) || !(rel_tol <= 1.0)) return FT_EINVAL;
    }
    const uintptr_t a = reinterpret_cast<uintptr_t>(ptr);
    std::lock_guard<std::mutex> lk(g_reg_mu);
    // no overlap with an area already registered
    auto next = g_reg.lower_bound(a);
    if (next != g_reg.end() && next->first < a + bytes) return FT_EINVAL;
    if (next != g_reg.begin()) {
        auto prev = std::prev(next);
        if (prev->first + prev->second.bytes > a) return FT_EINVAL;
    }
    g_reg[a] = Area{bytes, dtype, abs_tol, rel_tol};
    return FT_OK;
}

int ft_unregister_data(const void *ptr)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto it = g_reg.find(reinterpret_cast<uintptr_t>(ptr));
    if (it == g_reg.end()) return FT_ENOTFOUND;
    g_reg.erase(it);
    return FT_OK;
}

int ft_registered_type(const void *ptr, int32_t *dtype, double *abs_tol, double *rel_tol, uint64_t *bytes)
{
    std::lock_guard<std::mutex> lk(g_reg_mu);
    auto it = find_area(ptr);
    if (it == g_reg.end()) return FT_ENOTFOUND;
    const uintptr_t a = reinterpret_cast<uintptr_t>(ptr);
    if (dtype) *dtype = it->second.dtype;
    if (abs_tol) *abs_tol = it->second.abs_tol;
    if (rel_tol) *rel_tol = it->second.rel_tol;
    if (bytes) *bytes = it->first + it->second.bytes - a;   // from ptr to the area's end
    return FT_OK;
}

int ft_vote_registered(const void *const *replicas, int32_t R, void *out, uint32_t *block_crc, ft_stats *stats,
                       ft_stream stream)
{
    if (!replicas || R < 2 || R > FT_MAX_R) return FT_EINVAL;
    ft_vote_desc d;
    std::memset(&d, 0, sizeof(d));
    uint64_t bytes = 0;
    int rc = ft_registered_type(out, &d.dtype, &d.abs_tol, &d.rel_tol, &bytes);
    if (rc != FT_OK) return rc;
    for (int r = 0; r < R; ++r) d.replicas[r] = replicas[r];
    d.R = R;
    d.n = bytes / ftv::dtype_size(d.dtype);
    d.out = out;
    d.block_crc = block_crc;
    d.stats = stats;
    return ftv::vote_desc(&d, static_cast<cudaStream_t>(stream), nullptr);
}

int ft_dmr_run(ft_task_fn task, void *user, const ft_vote_desc *vote, ft_stream stream)
{
    if (!task || !vote) return FT_EINVAL;
    int rc = ftv::validate_desc(vote);
    if (rc != FT_OK) return rc;
    for (int r = 0; r < vote->R; ++r) {
        rc = task(user, r, const_cast<void *>(vote->replicas[r]), stream);
        if (rc != FT_OK) return rc;
    }
    return ftv::vote_desc(vote, static_cast<cudaStream_t>(stream), nullptr);
}

}  // extern "C"
