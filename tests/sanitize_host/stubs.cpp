// Stand-ins for the kernel launchers, so that the host code (tables, C ABI) links and runs under
// the sanitizers without a GPU.  Each returns MCPD_ECUDA; the host tests never reach them.
#include "mcpd.h"
#include "mcpd_internal.h"
namespace mcpd {
int pairs_shape(int, int, int, bool, size_t, int, size_t, long long, int, int, bool, bool, PairsShape *) { return MCPD_ECUDA; }
int pairs_y_regions(int, int) { return 0; }
size_t pairs_smem_bytes(size_t, int, int, int) { return 0; }
int batch_kernel_degree(int, int, int) { return 0; }
int launch_batch(const BParams &, int, int, size_t, void *) { return MCPD_ECUDA; }
int launch_group(const BParams &, int, int, size_t, void *) { return MCPD_ECUDA; }
int launch_pairs(const KParams &, int, int, size_t, void *) { return MCPD_ECUDA; }
int launch_philox(const uint32_t *, uint32_t, uint32_t, uint32_t *, long long, void *) { return MCPD_ECUDA; }
int pairs_max_smem(int, size_t *) { return MCPD_ECUDA; }
int set_group_smem(int, size_t) { return MCPD_ECUDA; }
int group_occupancy(int, int, size_t, int *) { return MCPD_ECUDA; }
int launch_finalize(const unsigned long long *, const unsigned long long *, const unsigned long long *, int, int, long long, long long, double *, double *, void *) { return MCPD_ECUDA; }
int group_max_threads(int) { return 0; }
int launch_finalize_batch(const InstDesc *, int, const int *, const int *, long long, double *, double *, void *) { return MCPD_ECUDA; }
}
extern "C" int mcpd_decode_noalloc(mcpd_ctx *, const mcpd_design *, const uint8_t *, const mcpd_params *, double *, double *, mcpd_stats *) { return MCPD_ECUDA; }
