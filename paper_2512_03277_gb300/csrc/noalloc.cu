// Allocation-free variant of the field-and-kick kernel (cavmd_field_kick_noalloc in cavmd.h).
//
// Some callers cannot allocate device memory once they are running: a framework that owns every
// byte of the GPU through its own pool (a cudaMalloc behind its back breaks its accounting and can
// fail when the pool has taken the free memory), a latency-critical loop where cudaMalloc and
// cudaFree would synchronise the device, or a plug-in whose host code is not allowed to allocate.
// For them this entry point keeps its only scratch, the per-block kinetic-energy partials and the
// last-block counter, in the file-scope array below, of fixed size. Every GPU that loads the
// library holds it until the process exits.
//
// The kernel is the same computation as the field kernel of a time step: E_n = sum_a U[a][n] W_a,
// p_j += tau F_j + E_n b_j for every atom of cell n, and the total kinetic energy after the kick,
// summed in a fixed order (per block, then by the last block to finish, block by block).
#include <mutex>
#include <string>

#include "cavmd_internal.cuh"

namespace {

constexpr int NA_CELLS = 32;
constexpr int NA_SLICES = 32;
constexpr int NA_MAX_BLOCKS = CAVMD_NOALLOC_MAX_CELLS / NA_CELLS;

// partials [0, NA_MAX_BLOCKS), then one slot whose first word is the last-block counter
static __device__ __align__(256) double noalloc_scratch[NA_MAX_BLOCKS + 32];

__global__ void __launch_bounds__(NA_CELLS *NA_SLICES)
k_field_kick_noalloc(int N, int M, const int *__restrict__ off, const double *__restrict__ U,
                     const double *__restrict__ W, const double *__restrict__ F,
                     const double *__restrict__ b, const double *__restrict__ inv_mass, double tau,
                     double *__restrict__ p, double *__restrict__ E_out, double *__restrict__ e_kin,
                     double *__restrict__ scratch) {
    __shared__ double red[NA_SLICES][NA_CELLS];
    __shared__ bool last;
    unsigned *counter = reinterpret_cast<unsigned *>(scratch + NA_MAX_BLOCKS);
    const int cl = threadIdx.x & (NA_CELLS - 1);
    const int sl = threadIdx.x / NA_CELLS;
    const int n = blockIdx.x * NA_CELLS + cl;
    double e = 0.0;
    if (n < N) {
        const double *u = U + n;
#pragma unroll 8
        for (int al = sl; al < M; al += NA_SLICES) e = fma(u[(size_t)al * N], __ldg(W + al), e);
    }
    red[sl][cl] = e;
    __syncthreads();
    double kin = 0.0;
    if (sl == 0 && n < N) {
        for (int s = 1; s < NA_SLICES; ++s) e += red[s][cl];
        if (E_out) E_out[n] = e;
        for (int j = off[n]; j < off[n + 1]; ++j) {
            const double im = inv_mass[j];
            for (int k = 0; k < 3; ++k) {
                const double pj = fma(tau, F[3 * j + k], fma(e, b[3 * j + k], p[3 * j + k]));
                p[3 * j + k] = pj;
                kin = fma(0.5 * im * pj, pj, kin);
            }
        }
    }
    if (sl == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) kin += __shfl_xor_sync(CAVMD_FULL_MASK, kin, o);
        if (cl == 0) {
            scratch[blockIdx.x] = kin;
            __threadfence();
            last = (atomicAdd(counter, 1u) == gridDim.x - 1);
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int i = threadIdx.x; i < (int)gridDim.x; i += blockDim.x) v += __ldcg(scratch + i);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(CAVMD_FULL_MASK, v, o);
    if (cl == 0) red[0][sl] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < NA_SLICES; ++w) t += red[0][w];
        *e_kin = t;
        *counter = 0u;
    }
}

// Device address of the scratch array per device, from the last lookup made outside a stream
// capture. Every call outside a capture looks the address up again (cheap), so a module reloaded
// after cudaDeviceReset is seen; a call during a capture uses the remembered address.
std::mutex g_mu;
void *g_scratch_addr[64] = {nullptr};

}  // namespace

extern "C" int cavmd_field_kick_noalloc(int32_t n_cells, int32_t n_modes, const int32_t *cell_offset,
                                        const double *U, const double *W, const double *F,
                                        const double *b, const double *inv_mass, double tau,
                                        double *p, double *E_out, double *e_kin_out, void *stream) {
    if (n_cells < 1 || n_cells > CAVMD_NOALLOC_MAX_CELLS) {
        cavmd_set_global_error("cavmd_field_kick_noalloc: n_cells must be in 1.." +
                               std::to_string(CAVMD_NOALLOC_MAX_CELLS) + ", got " + std::to_string(n_cells));
        return CAVMD_ERR_INVALID_ARG;
    }
    if (n_modes < 0 || !cell_offset || (n_modes > 0 && (!U || !W)) || !F || !b || !inv_mass || !p ||
        !e_kin_out) {
        cavmd_set_global_error("cavmd_field_kick_noalloc: NULL array or negative n_modes");
        return CAVMD_ERR_INVALID_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= 64) {
        cavmd_set_global_error(std::string("cavmd_field_kick_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
        return CAVMD_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) {
        cavmd_set_global_error(std::string("cavmd_field_kick_noalloc: cudaStreamIsCapturing: ") +
                               cudaGetErrorString(e));
        return CAVMD_ERR_CUDA;
    }
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (cap == cudaStreamCaptureStatusNone) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, noalloc_scratch);
            if (e != cudaSuccess) {
                cavmd_set_global_error(std::string("cavmd_field_kick_noalloc: cudaGetSymbolAddress: ") +
                                       cudaGetErrorString(e));
                return CAVMD_ERR_CUDA;
            }
            g_scratch_addr[dev] = ptr;
        } else if (!g_scratch_addr[dev]) {
            cavmd_set_global_error("cavmd_field_kick_noalloc: the first call on a device must come before any "
                                   "stream capture");
            return CAVMD_ERR_INVALID_ARG;
        }
        scratch = g_scratch_addr[dev];
    }
    // the last-block counter must start at zero
    e = cudaMemsetAsync(static_cast<double *>(scratch) + NA_MAX_BLOCKS, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) {
        cavmd_set_global_error(std::string("cavmd_field_kick_noalloc: cudaMemsetAsync: ") + cudaGetErrorString(e));
        return CAVMD_ERR_CUDA;
    }
    const int blocks = (n_cells + NA_CELLS - 1) / NA_CELLS;
    k_field_kick_noalloc<<<blocks, NA_CELLS * NA_SLICES, 0, st>>>(
        n_cells, n_modes, cell_offset, U, W, F, b, inv_mass, tau, p, E_out, e_kin_out,
        static_cast<double *>(scratch));
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        cavmd_set_global_error(std::string("cavmd_field_kick_noalloc: launch: ") + cudaGetErrorString(e));
        return CAVMD_ERR_CUDA;
    }
    return CAVMD_OK;
}
