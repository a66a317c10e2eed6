// sgtv_noalloc.cu -- the KKT residual of a given state without any device
// allocation, for callers that cannot call cudaMalloc (for example code that
// runs while a stream is being captured into a CUDA graph, under an external
// memory budget, or from a real-time loop that must not touch the allocator).
//
// The residual needs scratch beyond its inputs and outputs: the ratio
// y / (A f + r) (one value per measurement), the backprojection A^T ratio (one
// per hyper-voxel) and the per-block FP64 partials of the reduction. Here that
// scratch is one file-scope __device__ array of fixed size, which every GPU
// that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/sgtv.h"
#include "sgtv_internal.h"

using namespace sgtv;

namespace {

constexpr int64_t kMaxI = SGTV_NOALLOC_MAX_I;
constexpr int64_t kMaxJ = SGTV_NOALLOC_MAX_J;
constexpr int kPartBlocks = 1024;  // reduction blocks (two FP64 fields each)

// The scratch: ratio [kMaxI] and backprojection [kMaxJ] as FP32, the
// partials, then the one-scan geometry table the kernels read.
constexpr size_t kVecBytes = sizeof(float) * size_t(kMaxI + kMaxJ);
constexpr size_t kPartBytes = sizeof(double) * 2 * kPartBlocks;
constexpr size_t kGeomBytes = 256;
constexpr size_t kScratchBytes = kVecBytes + kPartBytes + kGeomBytes;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch, looked up once per device with that device
// current (the host-side name is only a stand-in for the symbol).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};

thread_local std::string g_err;

int reject(int code, const std::string &msg)
{
    g_err = msg;
    return code;
}

// Writes the geometry table of one scan into the scratch (no host copy).
__global__ void k_noalloc_geom(Scan *tab, int64_t *voff, int64_t *soff, int32_t Nx, int32_t Nz, int32_t Nq,
                               double rho)
{
    tab->vox0 = 0;
    tab->site0 = 0;
    tab->Nx = Nx;
    tab->Nz = Nz;
    tab->Nq = Nq;
    tab->pad_ = 0;
    tab->rho = rho;
    tab->tau = 0.0;
    tab->beta = 0.0;
    voff[0] = 0;
    voff[1] = int64_t(Nx) * Nz * Nq;
    soff[0] = 0;
    soff[1] = int64_t(Nx) * Nz;
}

}  // namespace

extern "C" {

const char *sgtv_noalloc_last_error(void) { return g_err.c_str(); }

int sgtv_kkt_residual_noalloc(int64_t I, int64_t J, const int64_t *csr_rowptr, const int32_t *csr_col,
                              const float *csr_val, const int64_t *csc_colptr, const int32_t *csc_row,
                              const float *csc_val, int32_t Nx, int32_t Nz, int32_t Nq, int32_t n_dirs,
                              const double *w, const float *y, const float *b, int64_t b_len, const float *s,
                              const float *f, const float *c, double rho, double *out, void *stream)
{
    g_err.clear();
    if (!csr_rowptr || !csr_col || !csr_val || !csc_colptr || !csc_row || !csc_val || !w || !y || !b || !s ||
        !f || !c || !out)
        return reject(SGTV_ERR_ARG, "a required pointer is NULL");
    if (I < 1 || J < 1) return reject(SGTV_ERR_ARG, "I and J must be >= 1");
    if (I > kMaxI || J > kMaxJ)
        return reject(SGTV_ERR_ARG, "I or J exceeds the fixed scratch of this entry point (I <= " +
                                        std::to_string(kMaxI) + ", J <= " + std::to_string(kMaxJ) + ")");
    if (Nx < 1 || Nz < 1 || Nq < 1 || int64_t(Nx) * Nz * Nq != J) return reject(SGTV_ERR_ARG, "J != Nx * Nz * Nq");
    if (n_dirs != 4 && n_dirs != 2) return reject(SGTV_ERR_ARG, "n_dirs must be 4 or 2");
    if (b_len != 1 && b_len != I) return reject(SGTV_ERR_ARG, "b_len must be 1 or I");

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return reject(SGTV_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return reject(SGTV_ERR_ARG, "device ordinal out of range");
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_addr[dev]) {
            e = cudaGetSymbolAddress(&g_addr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_addr[dev] = nullptr;
                return reject(SGTV_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
            }
        }
        scratch = g_addr[dev];
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return reject(SGTV_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));

    // Every scratch element read below is written first in the same call
    // (ratio by the forward projection, the backprojection by its kernel, each
    // partial by its block), so nothing needs clearing between calls.
    Dev d{};
    d.I = I;
    d.J = J;
    d.rowptr = csr_rowptr;
    d.colptr = csc_colptr;
    d.col = csr_col;
    d.row = csc_row;
    d.rval = csr_val;
    d.cval = csc_val;
    d.y = y;
    d.r = b;
    d.r_scalar = b_len == 1;
    d.s = const_cast<float *>(s);
    d.ratio = static_cast<float *>(scratch);
    d.e = static_cast<float *>(scratch) + kMaxI;
    d.c = const_cast<float *>(c);
    d.part = reinterpret_cast<double *>(static_cast<unsigned char *>(scratch) + kVecBytes);
    d.red = out;
    d.sm_count = sms;
    d.red_blocks = 2 * sms < kPartBlocks ? 2 * sms : kPartBlocks;
    unsigned char *geom = static_cast<unsigned char *>(scratch) + kVecBytes + kPartBytes;
    Scan *tab = reinterpret_cast<Scan *>(geom);
    int64_t *voff = reinterpret_cast<int64_t *>(geom + 128);
    int64_t *soff = voff + 2;
    Geom g{};
    g.n_dirs = n_dirs;
    g.nscans = 1;
    g.J = J;
    g.S = int64_t(Nx) * Nz;
    g.scans = tab;
    g.vox_off = voff;
    g.site_off = soff;
    static const int dx4[4] = {+1, -1, 0, 0}, dz4[4] = {0, 0, +1, -1};
    static const int dx2[4] = {+1, 0, 0, 0}, dz2[4] = {0, +1, 0, 0};
    for (int p = 0; p < 4; p++) {
        g.dx[p] = n_dirs == 4 ? dx4[p] : dx2[p];
        g.dz[p] = n_dirs == 4 ? dz4[p] : dz2[p];
        g.w[p] = p < n_dirs ? w[p] : 0.0;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    k_noalloc_geom<<<1, 1, 0, st>>>(tab, voff, soff, Nx, Nz, Nq, rho);
    const KernelSet &ks = kset_f32;
    ks.fwd[0](d, f, d.ratio, st);        // ratio = y / (A f + r), plain one-row-per-warp form
    ks.backproject(d, d.ratio, d.e, st); // e = A^T ratio
    ks.kkt(d, g, f, 0, st);              // out[0] = max |min(f, g)|, out[1] = max s (rho from the table)
    e = cudaGetLastError();
    if (e != cudaSuccess) return reject(SGTV_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
    return SGTV_OK;
}

}  // extern "C"
