// Compute entry points of libgint (C ABI), small helper kernels (block symmetrisation,
// FP64 reductions) and precision dispatch.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gint_device.cuh"

using namespace gint;

namespace gint {
cudaError_t launch_mirror(const Plan &P, double *H, cudaStream_t s);

gint_status check_handle(gint_handle h, const char *who)
{
    if (!h) {
        set_error("%s: null handle", who);
        return GINT_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (dev != h->device) {
        set_error("%s: current device %d differs from the handle's device %d", who, dev, h->device);
        return GINT_EINVAL;
    }
    return GINT_OK;
}


SInfo sinfo_for(const gint_handle_s *h, const double *V, double *H, const void *DMS, double *rho, double *F)
{
    SInfo si{};
    si.V = V;
    si.H = H;
    si.DMS = DMS;
    si.dms_plane = h->dms_plane;
    si.padn = h->bs[1].padn ? 1 : 0;
    si.rho = rho;
    si.F = F;
    si.poff = h->d_poff;
    for (int i = 0; i < 3; ++i) si.grid[i] = h->grid[i];
    si.dV = h->info.dV;
    si.phimax = h->phimax;
    si.amax = h->d_amax;
    for (int i = 0; i < 9; ++i) si.hstep[i] = (float)h->plan.h[i];
    return si;
}
}

namespace {

// DMs <- (DM + DM^T_block) / 2, DM^T_block(I,J,R) = DM(J,I,-R)^T
__global__ void k_symmetrise(Plan P, const double *__restrict__ DM, double *out)
{
    for (int64_t b = blockIdx.x; b < P.nblocks; b += gridDim.x) {
        const int pb = P.partner[b];
        const int64_t off = P.blk_off[b], poff = P.blk_off[pb];
        const int rows = P.blk_rows[b];
        const int cols = (int)((P.blk_off[b + 1] - off) / rows);
        for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
            const int mu = e / cols, nu = e - mu * cols;
            out[off + e] = 0.5 * (DM[off + e] + DM[poff + nu * rows + mu]);
        }
    }
}

// the largest of m over the threads of a block into *out (float bits of non-negative values
// order like unsigned integers)
__device__ __forceinline__ void block_max_to(float m, float *out)
{
    __shared__ float wm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wm[w]);
        atomicMax(reinterpret_cast<unsigned *>(out), __float_as_uint(b));
    }
}

// *out <- max(*out, max_i |x_i|) (FP32, rounded to nearest)
__global__ void k_absmax(const double *__restrict__ x, int64_t n, float *out)
{
    float m = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(d2f(x[i])));
    block_max_to(m, out);
}

__global__ void k_scale(double *x, int64_t n, double a)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        x[i] *= a;
}

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

// Deterministic two-pass FP64 reduction: block partials into scratch, then one block sums
// them in a fixed order.
__global__ void k_dot_partial(const double *__restrict__ a, const double *__restrict__ b, int64_t n, double *part)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        acc += b ? a[i] * b[i] : a[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

__global__ void k_dot_final(const double *part, int n, double scale, double *out)
{
    __shared__ double sh[kRedThreads];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) acc += part[i];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0] * scale;
}


bool valid_prec(gint_prec p) { return p >= GINT_FP64 && p <= GINT_FP16X3; }

gint_status do_dot(gint_handle h, const double *a, const double *b, int64_t n, double scale, double *out,
                   cudaStream_t s, const char *who)
{
    int nblk = (int)std::min<int64_t>(kRedBlocks, std::max<int64_t>(1, (n + kRedThreads - 1) / kRedThreads));
    k_dot_partial<<<nblk, kRedThreads, 0, s>>>(a, b, n, h->d_red);
    k_dot_final<<<1, kRedThreads, 0, s>>>(h->d_red, nblk, scale, out);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GINT_OK : cuda_fail(e, who);
}

gint_status run_vlocal(gint_handle h, const double *V, double *H, gint_prec prec, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(H, 0, sizeof(double) * h->info.nvalues, s);
    if (e != cudaSuccess) return cuda_fail(e, "gint_vlocal: memset");
    if (prec == GINT_FP16X3 && ((e = cudaMemsetAsync(h->d_amax, 0, sizeof(float), s)) != cudaSuccess ||
                                (e = launch_absmax(V, h->info.npts, h->d_amax, s)) != cudaSuccess))
        return cuda_fail(e, "gint_vlocal: potential range");
    if (prec == GINT_FP64 || prec == GINT_FP32)
        e = launch_vlocal_simt(plan_for(h, 0), prec == GINT_FP64, V, H, s, h->nsm);
    else
        e = launch_vlocal_tc(plan_for(h, 0), prec, sinfo_for(h, V, H, nullptr, nullptr, nullptr), nullptr, s, h->nsm,
                             h->bs[0].max_nb);
    if (e != cudaSuccess) return cuda_fail(e, "gint_vlocal: launch");
    e = launch_mirror(h->plan, H, s);
    if (e != cudaSuccess) return cuda_fail(e, "gint_vlocal: mirror");
    h->last_stream = s;
    return GINT_OK;
}

gint_status run_rho_force(gint_handle h, const double *V, const double *DM, double *rho, double *F, gint_prec prec,
                          cudaStream_t s, double *dLde = nullptr)
{
    cudaError_t e;
    const bool simt = (prec == GINT_FP64 || prec == GINT_FP32);
    const bool grad = F || dLde;   // derivatives use the block-symmetric part of the DM
    if (F && (e = cudaMemsetAsync(F, 0, sizeof(double) * 3 * h->natoms, s)) != cudaSuccess)
        return cuda_fail(e, "gint_force: memset");
    if (dLde && (e = cudaMemsetAsync(dLde, 0, sizeof(double) * 9, s)) != cudaSuccess)
        return cuda_fail(e, "gint_strain: memset");
    if (simt) {
        // CUDA-core kernels read FP64
        const double *D = DM;
        if (grad && h->info.nblocks > 0) {
            k_symmetrise<<<(int)std::min<int64_t>(h->info.nblocks, 8192), 128, 0, s>>>(h->plan, DM, h->d_dmsym);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gint_force: symmetrise");
            D = h->d_dmsym;
        }
        e = launch_rho_force_simt(plan_for(h, 1), prec == GINT_FP64, V, D, rho, F, dLde, s, h->nsm);
    } else {
        // tensor-core kernels copy the density matrix from its pre-split padded store
        float *amax = prec == GINT_FP16X3 ? h->d_amax + 1 : nullptr;
        if (amax && ((e = cudaMemsetAsync(amax, 0, sizeof(float), s)) != cudaSuccess ||
                     (e = launch_absmax(DM, h->info.nvalues, amax, s)) != cudaSuccess))
            return cuda_fail(e, "gint_rho: range");
        if (h->info.nvalues > 0 &&
            (e = launch_dm_split(h->plan, prec, (const int *)h->d_soff, DM, h->d_dms, h->dms_plane, h->bs[1].padn, grad,
                                 amax, s)) !=
                cudaSuccess)
            return cuda_fail(e, "gint_rho: split");
        SInfo si = sinfo_for(h, V, nullptr, h->d_dms, rho, F);
        si.dLde = dLde;
        e = launch_rho_force_tc(plan_for(h, 1), prec, si, nullptr, rho != nullptr, grad, s, h->nsm);
    }
    if (e != cudaSuccess) return cuda_fail(e, "gint_rho_force: launch");
    h->last_stream = s;
    return GINT_OK;
}

}  // namespace

extern "C" gint_status gint_vlocal(gint_handle h, const double *V_dev, double *H_dev, gint_prec prec, void *stream)
{
    gint_status st = check_handle(h, "gint_vlocal");
    if (st != GINT_OK) return st;
    if (!V_dev || !H_dev || !valid_prec(prec)) {
        set_error("gint_vlocal: null buffer or invalid precision");
        return GINT_EINVAL;
    }
    return run_vlocal(h, V_dev, H_dev, prec, (cudaStream_t)stream);
}

extern "C" gint_status gint_rho(gint_handle h, const double *DM_dev, double *rho_dev, gint_prec prec, void *stream)
{
    gint_status st = check_handle(h, "gint_rho");
    if (st != GINT_OK) return st;
    if (!DM_dev || !rho_dev || !valid_prec(prec)) {
        set_error("gint_rho: null buffer or invalid precision");
        return GINT_EINVAL;
    }
    return run_rho_force(h, nullptr, DM_dev, rho_dev, nullptr, prec, (cudaStream_t)stream);
}

extern "C" gint_status gint_force(gint_handle h, const double *V_dev, const double *DM_dev, double *F_dev,
                                  gint_prec prec, void *stream)
{
    gint_status st = check_handle(h, "gint_force");
    if (st != GINT_OK) return st;
    if (!V_dev || !DM_dev || !F_dev || !valid_prec(prec)) {
        set_error("gint_force: null buffer or invalid precision");
        return GINT_EINVAL;
    }
    return run_rho_force(h, V_dev, DM_dev, nullptr, F_dev, prec, (cudaStream_t)stream);
}

extern "C" gint_status gint_rho_force(gint_handle h, const double *V_dev, const double *DM_dev, double *rho_dev,
                                      double *F_dev, gint_prec prec, void *stream)
{
    gint_status st = check_handle(h, "gint_rho_force");
    if (st != GINT_OK) return st;
    if (!DM_dev || (!rho_dev && !F_dev) || (F_dev && !V_dev) || !valid_prec(prec)) {
        set_error("gint_rho_force: null buffer or invalid precision");
        return GINT_EINVAL;
    }
    return run_rho_force(h, V_dev, DM_dev, rho_dev, F_dev, prec, (cudaStream_t)stream);
}

extern "C" gint_status gint_strain_derivative(gint_handle h, const double *V_dev, const double *DM_dev,
                                              double *dLde_dev, gint_prec prec, void *stream)
{
    gint_status st = check_handle(h, "gint_strain_derivative");
    if (st != GINT_OK) return st;
    if (!V_dev || !DM_dev || !dLde_dev || !valid_prec(prec)) {
        set_error("gint_strain_derivative: null buffer or invalid precision");
        return GINT_EINVAL;
    }
    return run_rho_force(h, V_dev, DM_dev, nullptr, nullptr, prec, (cudaStream_t)stream, dLde_dev);
}

extern "C" gint_status gint_vlocal_backward(gint_handle h, const double *V_dev, const double *gH_dev, double *gV_dev,
                                            double *gtau_dev, gint_prec prec, void *stream)
{
    gint_status st = check_handle(h, "gint_vlocal_backward");
    if (st != GINT_OK) return st;
    if (!gH_dev || (!gV_dev && !gtau_dev) || (gtau_dev && !V_dev) || !valid_prec(prec)) {
        set_error("gint_vlocal_backward: null buffer or invalid precision");
        return GINT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = run_rho_force(h, V_dev, gH_dev, gV_dev, gtau_dev, prec, s)) != GINT_OK) return st;
    // rho -> dV rho, F -> -F (dL/dtau)
    if (gV_dev)
        k_scale<<<(int)std::min<int64_t>(4096, (h->info.npts + 255) / 256), 256, 0, s>>>(gV_dev, h->info.npts, h->info.dV);
    if (gtau_dev) k_scale<<<1, 256, 0, s>>>(gtau_dev, 3 * (int64_t)h->natoms, -1.0);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GINT_OK : cuda_fail(e, "gint_vlocal_backward: scale");
}

extern "C" gint_status gint_charge(gint_handle h, const double *rho_dev, double *out_dev, void *stream)
{
    gint_status st = check_handle(h, "gint_charge");
    if (st != GINT_OK) return st;
    if (!rho_dev || !out_dev) {
        set_error("gint_charge: null buffer");
        return GINT_EINVAL;
    }
    return do_dot(h, rho_dev, nullptr, h->info.npts, h->info.dV, out_dev, (cudaStream_t)stream, "gint_charge");
}

extern "C" gint_status gint_block_dot(gint_handle h, const double *A_dev, const double *B_dev, double *out_dev,
                                      void *stream)
{
    gint_status st = check_handle(h, "gint_block_dot");
    if (st != GINT_OK) return st;
    if (!A_dev || !B_dev || !out_dev) {
        set_error("gint_block_dot: null buffer");
        return GINT_EINVAL;
    }
    return do_dot(h, A_dev, B_dev, h->info.nvalues, 1.0, out_dev, (cudaStream_t)stream, "gint_block_dot");
}

extern "C" gint_status gint_run_host(gint_handle h, const double *V_host, const double *DM_host, double *H_host,
                                     double *rho_host, double *F_host, gint_prec prec, void *stream)
{
    gint_status st = check_handle(h, "gint_run_host");
    if (st != GINT_OK) return st;
    if (!V_host || !DM_host || !valid_prec(prec)) {
        set_error("gint_run_host: null input or invalid precision");
        return GINT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nv = (size_t)h->info.nvalues, np = (size_t)h->info.npts, na = (size_t)h->natoms;
    const size_t need = sizeof(double) * (2 * np + 2 * nv + 3 * na);
    cudaError_t e;
    if (h->hostio_bytes < need) {
        if (h->d_hostio) cudaFree(h->d_hostio);
        h->d_hostio = nullptr;
        h->hostio_bytes = 0;
        if ((e = cudaMalloc((void **)&h->d_hostio, need)) != cudaSuccess) return cuda_fail(e, "gint_run_host: allocate");
        h->hostio_bytes = need;
    }
    if (!h->io_stream) {
        if ((e = cudaStreamCreateWithFlags(&h->io_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "gint_run_host: copy stream");
        for (cudaEvent_t &ev : h->io_ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(e, "gint_run_host: events");
    }
    // The density matrix comes in on the copy stream while vlocal runs, and H goes out on it
    // while rho and the force run; V in and rho out stay on the critical path.
    cudaStream_t c = h->io_stream;
    cudaEvent_t v_in = h->io_ev[0], dm_in = h->io_ev[1], h_done = h->io_ev[2], h_out = h->io_ev[3];
    double *dV = h->d_hostio, *drho = dV + np, *dDM = drho + np, *dH = dDM + nv, *dF = dH + nv;
    if ((e = cudaEventRecord(h_out, s)) != cudaSuccess || (e = cudaStreamWaitEvent(c, h_out, 0)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dV, V_host, sizeof(double) * np, cudaMemcpyHostToDevice, c)) != cudaSuccess ||
        (e = cudaEventRecord(v_in, c)) != cudaSuccess ||
        (e = cudaMemcpyAsync(dDM, DM_host, sizeof(double) * nv, cudaMemcpyHostToDevice, c)) != cudaSuccess ||
        (e = cudaEventRecord(dm_in, c)) != cudaSuccess || (e = cudaStreamWaitEvent(s, v_in, 0)) != cudaSuccess)
        return cuda_fail(e, "gint_run_host: copy in");
    if ((st = run_vlocal(h, dV, dH, prec, s)) != GINT_OK) return st;
    if ((e = cudaEventRecord(h_done, s)) != cudaSuccess || (e = cudaStreamWaitEvent(s, dm_in, 0)) != cudaSuccess)
        return cuda_fail(e, "gint_run_host: order");
    if ((st = run_rho_force(h, dV, dDM, drho, dF, prec, s)) != GINT_OK) return st;
    if ((e = cudaStreamWaitEvent(c, h_done, 0)) != cudaSuccess ||
        (H_host && (e = cudaMemcpyAsync(H_host, dH, sizeof(double) * nv, cudaMemcpyDeviceToHost, c)) != cudaSuccess) ||
        (e = cudaEventRecord(h_out, c)) != cudaSuccess ||
        (rho_host && (e = cudaMemcpyAsync(rho_host, drho, sizeof(double) * np, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (F_host && (e = cudaMemcpyAsync(F_host, dF, sizeof(double) * 3 * na, cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (e = cudaStreamWaitEvent(s, h_out, 0)) != cudaSuccess)
        return cuda_fail(e, "gint_run_host: copy out");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "gint_run_host: synchronise");
    return GINT_OK;
}

extern "C" gint_status gint_get_status(gint_handle h)
{
    gint_status st = check_handle(h, "gint_get_status");
    if (st != GINT_OK) return st;
    cudaError_t e = cudaStreamSynchronize(h->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "gint_get_status: synchronise");
    int w = 0;
    if ((e = cudaMemcpy(&w, h->d_status, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "gint_get_status: read");
    if (w != 0) {
        cudaMemset(h->d_status, 0, sizeof(int));
        set_error("a kernel gave up on a bounded wait (status %d)", w);
        return (gint_status)w;
    }
    return GINT_OK;
}


namespace gint {
cudaError_t launch_absmax(const double *x, int64_t n, float *out, cudaStream_t s)
{
    const int grid = (int)std::min<int64_t>((n + 255) / 256, 2048);
    if (grid < 1) return cudaSuccess;
    k_absmax<<<grid, 256, 0, s>>>(x, n, out);
    return cudaGetLastError();
}
}  // namespace gint
