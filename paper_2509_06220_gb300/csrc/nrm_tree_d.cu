// nrm_tree_d.cu -- the binary64 (D) tree kernels and their entry points
// (instantiated here from nrm_tree.cuh), and nrmf_d_noalloc.
#include "nrm_tree.cuh"

namespace nrm {

nrm_status run_single_x(nrm_ctx *c, const double *x, int64_t n, double p, double *out, cudaStream_t s,
                        int64_t item_lo, int64_t item_hi, const VecPlan *plan_in, int64_t stride, int variant) {
    return run_single<double>(c, x, n, p, out, s, item_lo, item_hi, plan_in, stride, variant);
}

nrm_status run_batch_x(nrm_ctx *c, const double *x, int64_t x_len, const int64_t *off, const int64_t *lens,
                       int64_t B, double p, const double *p_dev, double *out, int32_t *status, cudaStream_t s,
                       double *lanes) {
    return run_batch<double>(c, x, x_len, off, lens, B, p, p_dev, out, status, s, lanes);
}

} // namespace nrm

using namespace nrm;

// ---------------------------------------------------------------------------
// nrmf_d_noalloc: xNRMF in binary64 without any allocation.
//
// Some callers cannot call cudaMalloc: cudaMalloc and cudaFree can
// synchronise the whole device, which a latency-critical loop cannot
// afford, and some applications give all device memory to their own
// allocator or run under a fixed budget that forbids allocations outside it.
// This entry point therefore needs no context.  Its scratch (the tree's
// ticket counters and partial-norm slots) is the file-scope array below,
// created when the library is loaded onto a device and held until the
// process exits.  It is shared by every call on that device and keeps the
// last call's contents; the tickets are cleared on the stream at the start of
// each call.  The array's device address is looked up once per device; a
// cudaDeviceReset destroys the array with the context, after which this
// entry point must not be called again in the process.
// ---------------------------------------------------------------------------
namespace {

// Size limit: n <= 2^29 gives m <= 2^23 rows, a row tree of depth D <= 23,
// and with at most 2^11 work items each item holds k = D - dw <= 12 =
// NA_G + MAXL levels, the deepest the counter stack supports.
constexpr int NA_DW_MAX = 11;                                // at most 2^11 work items
constexpr int64_t NA_NODES = (int64_t(1) << NA_DW_MAX) - 1;  // internal tree nodes
constexpr size_t NA_TICKET_BYTES = 8192;                     // >= NA_NODES * 4, slot-aligned
constexpr size_t NA_SLOT_BYTES = (size_t)2 * NA_NODES * 512; // one 512-byte row per child node
constexpr int NA_G = 2, NA_WPB = 4;
static_assert(NA_TICKET_BYTES >= (size_t)NA_NODES * 4 && NA_TICKET_BYTES % 512 == 0, "ticket area");
static_assert(NA_DW_MAX + NA_G + MAXL >= 23, "n = 2^29 (2^23 rows) must fit the scratch and the stack");
constexpr int NA_MAX_DEVICES = 64;

static __device__ __align__(256) unsigned char nrm_noalloc_scratch[NA_TICKET_BYTES + NA_SLOT_BYTES];

struct NaDevice {
    bool ready = false;
    unsigned char *scratch = nullptr; // device address of nrm_noalloc_scratch
    int sms = 0;
    int occ = 1;
};
NaDevice na_devices[NA_MAX_DEVICES];
std::mutex na_mutex;

// One-time set-up per device, with that device current: look up the
// device address of the scratch array (host code cannot use the symbol
// itself) and the occupancy of the kernel.
nrm_status na_setup(int dev, NaDevice **out) {
    std::lock_guard<std::mutex> lock(na_mutex);
    NaDevice &d = na_devices[dev];
    if (!d.ready) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, nrm_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return NRM_ECUDA;
        }
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return NRM_ECUDA;
        int occ = 0;
        const size_t smem = tree_smem_bytes<NA_G, OpHypot<double>>(NA_WPB, MAXL);
        e = cudaFuncSetAttribute(tree_kernel<double, NA_G, OpHypot<double>>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return NRM_ECUDA;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, tree_kernel<double, NA_G, OpHypot<double>>,
                                                          NA_WPB * 32, smem);
        if (e != cudaSuccess) return NRM_ECUDA;
        d.occ = std::max(1, occ);
        d.scratch = static_cast<unsigned char *>(p);
        d.ready = true;
    }
    *out = &d;
    return NRM_OK;
}

} // namespace

extern "C" nrm_status nrmf_d_noalloc(const double *x, int64_t n, double *out, void *stream) {
    if (!out || n < 0 || (n > 0 && !x)) return NRM_EINVAL;
    if (n > NRM_NOALLOC_MAX_N) return NRM_EINVAL; // the tree would need more scratch than the array holds
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(double), s) == cudaSuccess ? NRM_OK : NRM_ECUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return NRM_EDEVICE;
    NaDevice *d = nullptr;
    nrm_status st = na_setup(dev, &d);
    if (st != NRM_OK) return st;

    // the same tree as nrmf_d; only the cut depth is capped by the scratch size
    VecPlan pl{};
    pl.n = n;
    pl.stride = 1;
    pl.m = (n + 63) / 64;
    pl.D = ceil_log2_i64(pl.m);
    int dw = std::max(pl.D - 7, ceil_log2_i64((int64_t)d->sms * NA_WPB * 2));
    dw = std::min(dw, pl.D - NA_G);
    dw = std::max(dw, 0);
    dw = std::min(dw, NA_DW_MAX);
    pl.dw = dw;
    pl.k = pl.D - dw;
    if (pl.k > NA_G + MAXL) return NRM_EINVAL;
    const int64_t items = int64_t(1) << dw;
    const int64_t nodes = items - 1;

    unsigned *tickets = reinterpret_cast<unsigned *>(d->scratch);
    double *slots = reinterpret_cast<double *>(d->scratch + NA_TICKET_BYTES);
    if (nodes > 0 && cudaMemsetAsync(tickets, 0, (size_t)nodes * sizeof(unsigned), s) != cudaSuccess)
        return NRM_ECUDA;
    TreeArgs<double> a{};
    a.x = x;
    a.out = out;
    a.plans = nullptr;
    a.one = pl;
    a.B = 1;
    a.item_lo = 0;
    a.item_hi = items;
    a.tickets = tickets;
    a.slots = slots;
    a.levels = MAXL;
    const size_t smem = tree_smem_bytes<NA_G, OpHypot<double>>(NA_WPB, MAXL);
    const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>((items + NA_WPB - 1) / NA_WPB,
                                                                  (int64_t)d->sms * d->occ));
    // the kernel's dynamic shared memory limit is a per-function attribute
    // that other entry points set for their own launches (possibly lower)
    if (cudaFuncSetAttribute(tree_kernel<double, NA_G, OpHypot<double>>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return NRM_ECUDA;
    tree_kernel<double, NA_G, OpHypot<double>><<<(unsigned)blocks, NA_WPB * 32, smem, s>>>(a, OpHypot<double>{});
    return cudaGetLastError() == cudaSuccess ? NRM_OK : NRM_ECUDA;
}
