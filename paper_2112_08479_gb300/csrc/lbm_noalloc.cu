// lbm_noalloc.cu -- diagnostics entry point that allocates nothing.
//
// Some callers cannot allocate device memory at all: code running inside an
// allocator callback or an out-of-memory handler, embedders whose memory pool
// is fixed before this library is loaded, or hosts that forbid cudaMalloc
// after start-up.  lbm_diag_static serves them: it computes the same
// front / friction / budget diagnostics as lbm_diag, but from a state the
// caller already holds (canonical layout) and with all of its scratch in the
// fixed device array below, so it needs no workspace and calls no
// cudaMalloc, cudaFree or allocating library routine.
//
// The array lives for as long as the library stays loaded, on every device
// the library is used on.  Every call shares it: two calls that overlap on
// the GPU (different streams, or different host threads on one device) race
// on it and give wrong results; serialise them.  Each call re-initialises
// the parts that must start from a known value (column maxima, error flags);
// the rest is fully overwritten before it is read.
#include <math.h>
#include <mutex>
#include <stdio.h>
#include <string.h>

#include "lbm_internal.h"

namespace {

using namespace lbmgpu;

constexpr int NA_BX = 128;              // threads per column block
constexpr int NA_FIN = 512;             // threads of the finalize block
constexpr int NA_MAX_NX = 16384;        // largest nx served
constexpr int NA_MAX_BLOCKS = 32768;    // largest ceil(nx / 128) * nz served
constexpr int NA_MAX_DEVICES = 64;

struct NaRecord {
    double front, front_node, Fw, mass_delta, scalar_mass;
    int flags, pad;
};

// Scratch layout (byte offsets, 256-aligned): column keys, per-block budget
// partials (2 doubles), per-block friction partials (2 floats), the record.
constexpr size_t NA_KEYS = 0;
constexpr size_t NA_PART = NA_KEYS + (size_t)NA_MAX_NX * sizeof(unsigned);
constexpr size_t NA_FWPART = NA_PART + (size_t)NA_MAX_BLOCKS * 2 * sizeof(double);
constexpr size_t NA_REC = NA_FWPART + (size_t)NA_MAX_BLOCKS * 2 * sizeof(float);
constexpr size_t NA_BYTES = NA_REC + 256;   // 851,968 + 256 bytes

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

__device__ __forceinline__ unsigned na_key(float v) {
    const unsigned b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float na_key_inv(unsigned k) {
    const unsigned b = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(b);
}
__device__ __forceinline__ void na_pair_add(float& s, float& c, float t, float d) {
    float r, e;
    two_sum(s, t, r, e);
    s = r;
    c = c + d + e;
}

__global__ void na_reset_kernel(unsigned char* scratch, int nx) {
    unsigned* keys = (unsigned*)(scratch + NA_KEYS);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nx) keys[i] = 0x007fffffu;  // key of -inf
    if (i == 0) ((NaRecord*)(scratch + NA_REC))->flags = 0;
}

// One thread per column (x, z) of a canonical state ([Q + NS][N] floats,
// f - w then Phi - w), looping over y: the same sums as the workspace-based
// diagnostics.
template <int Q, int NS>
__global__ void __launch_bounds__(NA_BX) na_columns_kernel(KParams kp, const float* __restrict__ s,
                                                           unsigned char* scratch) {
    unsigned* keys = (unsigned*)(scratch + NA_KEYS);
    double* part = (double*)(scratch + NA_PART);
    float* fwpart = (float*)(scratch + NA_FWPART);
    NaRecord* rec = (NaRecord*)(scratch + NA_REC);
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int z = blockIdx.y;
    const size_t N = kp.N;
    double m_rho = 0.0, m_chi = 0.0;
    float fs = 0.0f, fc = 0.0f;
    if (x < kp.nx) {
        Kahan kc, kr, ku;
        int bad = 0;
        for (int y = 0; y < kp.ny; ++y) {
            const size_t n = (size_t)x + (size_t)kp.nx * ((size_t)y + (size_t)kp.ny * z);
            float c = 0.0f, d = 0.0f, jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
            for (int k = 0; k < NS; ++k) c += s[(size_t)(Q + k) * N + n];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float v = s[(size_t)i * N + n];
                d += v;
                jx += cx27(i) * v;
                jy += cy27(i) * v;
                jz += cz27(i) * v;
            }
            const float irho = 1.0f / (1.0f + d);
            const float chi = 1.0f + c;
            const float ux = (jx + 0.5f * kp.gx * chi) * irho;
            const float uy = (jy + 0.5f * kp.gy * chi) * irho;
            const float uz = (jz + 0.5f * kp.gz * chi) * irho;
            kc.add(c);
            kr.add(d);
            ku.add(ux);
            if (!(1.0f + d > 0.0f)) bad |= LBM_DEVFLAG_RHO_NONPOS;
            if (!isfinite(d) || !isfinite(ux) || !isfinite(uy) || !isfinite(uz) || !isfinite(c))
                bad |= LBM_DEVFLAG_NONFINITE;
        }
        if (bad) atomicOr(&rec->flags, bad);
        const float cb = 1.0f + (kc.s + kc.c) / (float)kp.ny;
        atomicMax(keys + x, na_key(cb));
        m_rho = (double)kr.s + (double)kr.c;
        m_chi = (double)kc.s + (double)kc.c;
        if (kp.nz >= 2 && z < 2) {
            const float a = z == 0 ? 3.0f * kp.nu : -kp.nu * (1.0f / 3.0f);
            fs = a * ku.s;
            fc = a * ku.c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        m_rho += __shfl_down_sync(0xffffffffu, m_rho, o);
        m_chi += __shfl_down_sync(0xffffffffu, m_chi, o);
        const float ts = __shfl_down_sync(0xffffffffu, fs, o);
        const float tc = __shfl_down_sync(0xffffffffu, fc, o);
        na_pair_add(fs, fc, ts, tc);
    }
    __shared__ double sr[NA_BX / 32], sc[NA_BX / 32];
    __shared__ float ss[NA_BX / 32], se[NA_BX / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) { sr[wid] = m_rho; sc[wid] = m_chi; ss[wid] = fs; se[wid] = fc; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, b = 0.0;
        float t = 0.0f, c = 0.0f;
        for (int w = 0; w < NA_BX / 32; ++w) { a += sr[w]; b += sc[w]; na_pair_add(t, c, ss[w], se[w]); }
        const unsigned blk = blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * blk] = a;
        part[2 * blk + 1] = b;
        fwpart[2 * blk] = t;
        fwpart[2 * blk + 1] = c;
    }
}

__global__ void __launch_bounds__(NA_FIN) na_finalize_kernel(int nx, double nodes, unsigned nblocks,
                                                             unsigned char* scratch, double thr,
                                                             int x0, double H, int xlim) {
    const unsigned* keys = (const unsigned*)(scratch + NA_KEYS);
    const double* part = (const double*)(scratch + NA_PART);
    const float* fwpart = (const float*)(scratch + NA_FWPART);
    NaRecord* rec = (NaRecord*)(scratch + NA_REC);
    __shared__ double sa[NA_FIN], sb[NA_FIN];
    __shared__ float ss[NA_FIN], sc[NA_FIN];
    __shared__ int sx[NA_FIN];
    const int t = threadIdx.x;
    double a = 0.0, b = 0.0;
    float s = 0.0f, c = 0.0f;
    for (unsigned i = t; i < nblocks; i += NA_FIN) {
        a += part[2 * i];
        b += part[2 * i + 1];
        na_pair_add(s, c, fwpart[2 * i], fwpart[2 * i + 1]);
    }
    int xf = -1;
    for (int x = t; x < xlim; x += NA_FIN)
        if ((double)na_key_inv(keys[x]) >= thr) xf = x;
    sa[t] = a; sb[t] = b; ss[t] = s; sc[t] = c; sx[t] = xf;
    __syncthreads();
    for (int w = NA_FIN / 2; w > 0; w >>= 1) {
        if (t < w) {
            sa[t] += sa[t + w];
            sb[t] += sb[t + w];
            float s0 = ss[t], c0 = sc[t];
            na_pair_add(s0, c0, ss[t + w], sc[t + w]);
            ss[t] = s0; sc[t] = c0;
            sx[t] = max(sx[t], sx[t + w]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const int x = sx[0];
        double xn;
        if (x < 0) xn = -1.0;
        else if (x == xlim - 1) xn = (double)x;
        else {
            const double m0 = na_key_inv(keys[x]), m1 = na_key_inv(keys[x + 1]);
            xn = x + (m0 - thr) / (m0 - m1);
        }
        rec->front_node = xn;
        rec->front = (xn + 0.5 - x0) / H;
        rec->Fw = (double)ss[0] + (double)sc[0];
        rec->mass_delta = sa[0];
        rec->scalar_mass = nodes + sb[0];
    }
}

std::mutex g_na_mutex;
void* g_na_ptr[NA_MAX_DEVICES];   // device address of g_na_scratch, per device
}  // namespace

namespace lbmgpu {
void lbm_set_thread_error(const char* msg);
}

extern "C" {

lbm_status lbm_diag_static(const lbm_params* p, const float* state, int64_t step,
                           void* cuda_stream, lbm_diagnostics* out_host) {
    if (lbm_validate(p) != LBM_OK) return LBM_ERR_ARG;
    if (!state || !out_host) return LBM_ERR_ARG;
    const int nbx = (p->nx + NA_BX - 1) / NA_BX;
    if (p->nx > NA_MAX_NX || (long long)nbx * p->nz > NA_MAX_BLOCKS) {
        char msg[128];
        snprintf(msg, sizeof msg, "lbm_diag_static serves nx <= %d and ceil(nx/128)*nz <= %d",
                 NA_MAX_NX, NA_MAX_BLOCKS);
        lbmgpu::lbm_set_thread_error(msg);
        return LBM_ERR_ARG;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return LBM_ERR_CUDA;
    // the call ends with a stream synchronisation, which a stream under
    // capture does not allow: refuse before enqueueing anything
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing((cudaStream_t)cuda_stream, &cap)) != cudaSuccess)
        return LBM_ERR_CUDA;
    if (cap != cudaStreamCaptureStatusNone) {
        lbmgpu::lbm_set_thread_error("lbm_diag_static cannot run while its stream is captured");
        return LBM_ERR_ARG;
    }
    // the state must be device (or managed) memory of the current device
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, state) != cudaSuccess ||
        (pa.type != cudaMemoryTypeDevice && pa.type != cudaMemoryTypeManaged) ||
        (pa.type == cudaMemoryTypeDevice && pa.device != dev)) {
        cudaGetLastError();   // clear a lookup error of an unknown pointer
        lbmgpu::lbm_set_thread_error("lbm_diag_static: state is not memory of the current device");
        return LBM_ERR_ARG;
    }
    void* scratch;
    {
        // set-up, once per device, with that device current: the device
        // address of the scratch array (its name is only a host-side stand-in)
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_na_scratch);
            if (e != cudaSuccess || !ptr) return LBM_ERR_CUDA;
            g_na_ptr[dev] = ptr;
        }
        scratch = g_na_ptr[dev];
    }
    KParams kp;
    memset(&kp, 0, sizeof kp);
    kp.nx = p->nx; kp.ny = p->ny; kp.nz = p->nz; kp.flags = p->flags;
    kp.N = (unsigned)((size_t)p->nx * p->ny * p->nz);
    kp.nxny = (unsigned)((size_t)p->nx * p->ny);
    kp.gx = (float)(p->gprime * p->eg[0]);
    kp.gy = (float)(p->gprime * p->eg[1]);
    kp.gz = (float)(p->gprime * p->eg[2]);
    kp.nu = (float)p->nu;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    unsigned char* s8 = (unsigned char*)scratch;
    na_reset_kernel<<<(p->nx + 255) / 256, 256, 0, st>>>(s8, p->nx);
    dim3 grid(nbx, p->nz);
    if (p->model == LBM_CUMULANT_Q27) {
        if (p->scalar == LBM_SCALAR_Q27) na_columns_kernel<27, 27><<<grid, NA_BX, 0, st>>>(kp, state, s8);
        else na_columns_kernel<27, 7><<<grid, NA_BX, 0, st>>>(kp, state, s8);
    } else {
        if (p->scalar == LBM_SCALAR_Q6) na_columns_kernel<19, 6><<<grid, NA_BX, 0, st>>>(kp, state, s8);
        else na_columns_kernel<19, 7><<<grid, NA_BX, 0, st>>>(kp, state, s8);
    }
    na_finalize_kernel<<<1, NA_FIN, 0, st>>>(p->nx, (double)kp.N, (unsigned)(nbx * p->nz), s8,
                                             p->front_threshold, p->x0, (double)p->H,
                                             front_xlim(p->nx, p->x0, p->flags));
    if ((e = cudaGetLastError()) != cudaSuccess) return LBM_ERR_CUDA;
    NaRecord rec;
    e = cudaMemcpyAsync(&rec, s8 + NA_REC, sizeof rec, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return LBM_ERR_CUDA;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return LBM_ERR_CUDA;
    out_host->front = rec.front;
    out_host->front_node = rec.front_node;
    out_host->Fw = rec.Fw;
    out_host->mass_delta = rec.mass_delta;
    out_host->scalar_mass = rec.scalar_mass;
    out_host->step = step;
    out_host->flags = rec.flags;
    out_host->pad_ = 0;
    return rec.flags ? LBM_ERR_UNSTABLE : LBM_OK;
}

}  // extern "C"
