// lbm_slab.cu -- halo exchange of an x-slab decomposition of the box.
//
// A box of nx_global columns is cut along x into slabs, one per GPU.  Each
// slab runs the ordinary step kernels with walls at its two x ends; the
// exchange below turns those walls into fluid.  In the AA pattern (see
// lbm_common.cuh) a node at a slab face reads, for each population i whose
// upwind node lies in the neighbouring slab, its own slot i (what a wall
// would reflect) -- on odd steps in the step kernel, after even steps also
// in every read of the state -- and on odd steps it writes each population
// leaving across the face to its own slot opp(i).  So one swap after every
// step makes the slab behave as part of the whole box:
//
//   slot i of face node (y, z)  <-  slot opp(i) of the neighbour's face node
//                                   (y - c_iy, z - c_iz)
//
// for every population i whose c_ix points into the slab (c_ix = +1 at the
// face x = 0, -1 at x = nx - 1), y periodic, and only where z - c_iz lies
// inside the box (otherwise the population meets the top or bottom wall and
// the reflected value in the node's own slot is the right one).  After an
// even step this hands each face node the post-collision populations of its
// upwind neighbours across the face; after an odd step it hands each
// neighbour the populations the face node pushed across.  Both sides pack
// before either unpacks (a swap), since each unpack overwrites the slots the
// other side sends.
//
// Face buffer of one slab face: the face's populations with c_ix = +1 (face
// 0) or -1 (face 1), fluid directions in increasing index then scalar ones,
// each as nz x ny storage elements ([k][z][y], y fastest): what the
// neighbour's unpack reads.
#include "lbm_internal.h"

namespace lbmgpu {

namespace {

// Number of directions d in [d0, d0 + n) with c_x(d) = s, and the position
// of direction d among them.
__host__ __device__ constexpr int face_count(int d0, int n, int s) {
    int c = 0;
    for (int d = d0; d < d0 + n; ++d) c += cx27(d) == s;
    return c;
}
__host__ __device__ constexpr int face_pos(int d0, int d, int s) {
    int c = 0;
    for (int e = d0; e < d; ++e) c += cx27(e) == s;
    return c;
}

// FACE 0: x = 0, populations with c_x = +1; FACE 1: x = nx - 1, c_x = -1.
template <int Q, int SL, typename S, int FACE>
__global__ void halo_pack_kernel(KParams kp, const S* __restrict__ f, const S* __restrict__ phi,
                                 S* __restrict__ buf) {
    constexpr int s = FACE == 0 ? 1 : -1;
    constexpr int D0 = ScalarLat<SL>::D0, NS = ScalarLat<SL>::NS;
    constexpr int NF = face_count(0, Q, s);
    const unsigned nyz = (unsigned)kp.ny * kp.nz;
    const unsigned yz = blockIdx.x * blockDim.x + threadIdx.x;
    if (yz >= nyz) return;
    const unsigned y = yz % kp.ny, z = yz / kp.ny;
    const unsigned n = z * kp.nxny + y * kp.nx + (FACE == 0 ? 0u : (unsigned)kp.nx - 1u);
    const size_t N = kp.N;
    // extent of the face buffer, checked in the debug build
    const size_t nb = (size_t)(NF + face_count(D0, NS, s)) * nyz;
#pragma unroll
    for (int d = 0; d < Q; ++d) {
        if (cx27(d) != s) continue;
        const size_t o = (size_t)face_pos(0, d, s) * nyz + yz, i = (size_t)d * N + n;
        if (LBM_IN(kp, LBM_SITE_HALO, buf, buf + o, 1, nb) &&
            LBM_IN(kp, LBM_SITE_HALO, f, f + i, 1, (size_t)Q * N))
            buf[o] = f[i];
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        if (cx27(k + D0) != s) continue;
        const size_t o = (size_t)(NF + face_pos(D0, k + D0, s)) * nyz + yz, i = (size_t)k * N + n;
        if (LBM_IN(kp, LBM_SITE_HALO, buf, buf + o, 1, nb) &&
            LBM_IN(kp, LBM_SITE_HALO, phi, phi + i, 1, (size_t)NS * N))
            buf[o] = phi[i];
    }
}

// Writes the neighbour's face buffer (its populations with c_x = -s) into
// this face's populations with c_x = s, shifted by (c_y, c_z) as above.
template <int Q, int SL, typename S, int FACE>
__global__ void halo_unpack_kernel(KParams kp, S* __restrict__ f, S* __restrict__ phi,
                                   const S* __restrict__ nbuf) {
    constexpr int s = FACE == 0 ? 1 : -1;
    constexpr int D0 = ScalarLat<SL>::D0, NS = ScalarLat<SL>::NS;
    constexpr int NFN = face_count(0, Q, -s);   // fluid entries of the neighbour's buffer
    const bool pz = (kp.flags & LBM_FLAG_PERIODIC_Z) != 0;
    const unsigned nyz = (unsigned)kp.ny * kp.nz;
    const unsigned yz = blockIdx.x * blockDim.x + threadIdx.x;
    if (yz >= nyz) return;
    const int y = (int)(yz % kp.ny), z = (int)(yz / kp.ny);
    const unsigned n = (unsigned)z * kp.nxny + (unsigned)y * kp.nx +
                       (FACE == 0 ? 0u : (unsigned)kp.nx - 1u);
    const size_t N = kp.N;
    // buffer index of the neighbour's face node (y - cy, z - cz); false
    // beyond the top or bottom wall
    auto src = [&](int cy, int cz, unsigned& idx) -> bool {
        int ys = y - cy, zs = z - cz;
        ys = ys < 0 ? ys + kp.ny : (ys >= kp.ny ? ys - kp.ny : ys);
        if (zs < 0 || zs >= kp.nz) {
            if (!pz) return false;
            zs = zs < 0 ? zs + kp.nz : zs - kp.nz;
        }
        idx = (unsigned)zs * kp.ny + (unsigned)ys;
        return true;
    };
    // extent of the face buffer, checked in the debug build
    const size_t nb = (size_t)(NFN + face_count(D0, NS, -s)) * nyz;
#pragma unroll
    for (int d = 0; d < Q; ++d) {
        if (cx27(d) != s) continue;
        unsigned idx;
        if (!src(cy27(d), cz27(d), idx)) continue;
        const size_t o = (size_t)face_pos(0, opp(d), -s) * nyz + idx, i = (size_t)d * N + n;
        if (LBM_IN(kp, LBM_SITE_HALO, nbuf, nbuf + o, 1, nb) &&
            LBM_IN(kp, LBM_SITE_HALO, f, f + i, 1, (size_t)Q * N))
            f[i] = nbuf[o];
    }
#pragma unroll
    for (int k = 0; k < NS; ++k) {
        const int d = k + D0;
        if (cx27(d) != s) continue;
        unsigned idx;
        if (!src(cy27(d), cz27(d), idx)) continue;
        const size_t o = (size_t)(NFN + face_pos(D0, opp(d), -s)) * nyz + idx,
                     i = (size_t)k * N + n;
        if (LBM_IN(kp, LBM_SITE_HALO, nbuf, nbuf + o, 1, nb) &&
            LBM_IN(kp, LBM_SITE_HALO, phi, phi + i, 1, (size_t)NS * N))
            phi[i] = nbuf[o];
    }
}

template <int Q, int SL, typename S>
cudaError_t launch_face(const KParams& kp, int face, bool pack, void* f, void* phi, void* buf,
                        cudaStream_t st) {
    const unsigned nyz = (unsigned)kp.ny * kp.nz;
    const dim3 grid((nyz + 255) / 256), block(256);
    if (pack) {
        if (face == 0)
            halo_pack_kernel<Q, SL, S, 0><<<grid, block, 0, st>>>(kp, (const S*)f, (const S*)phi, (S*)buf);
        else
            halo_pack_kernel<Q, SL, S, 1><<<grid, block, 0, st>>>(kp, (const S*)f, (const S*)phi, (S*)buf);
    } else {
        if (face == 0)
            halo_unpack_kernel<Q, SL, S, 0><<<grid, block, 0, st>>>(kp, (S*)f, (S*)phi, (const S*)buf);
        else
            halo_unpack_kernel<Q, SL, S, 1><<<grid, block, 0, st>>>(kp, (S*)f, (S*)phi, (const S*)buf);
    }
    return cudaGetLastError();
}

template <int Q, int SL>
cudaError_t launch_face_storage(const KParams& kp, int storage, int face, bool pack, void* f,
                                void* phi, void* buf, cudaStream_t st) {
    switch (storage) {
        case LBM_FP32: return launch_face<Q, SL, float>(kp, face, pack, f, phi, buf, st);
        case LBM_FP16S: return launch_face<Q, SL, __half>(kp, face, pack, f, phi, buf, st);
        case LBM_BF16S: return launch_face<Q, SL, __nv_bfloat16>(kp, face, pack, f, phi, buf, st);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

// Storage elements of one face buffer: the populations with c_x = +1 (the
// same count as -1) of both lattices, times ny nz.
size_t halo_elems(int Q, int NS, int ny, int nz) {
    const int nf = face_count(0, Q, 1);
    const int ns = NS == 6 ? face_count(1, 6, 1) : face_count(0, NS, 1);
    return (size_t)(nf + ns) * ny * nz;
}

cudaError_t launch_halo(const KParams& kp, Kind k, int face, bool pack, void* f, void* phi,
                        void* buf, cudaStream_t st) {
    if (k.model == LBM_BGK_SMAG_Q19 && k.scalar == LBM_SCALAR_Q7)
        return launch_face_storage<19, 7>(kp, k.storage, face, pack, f, phi, buf, st);
    if (k.model == LBM_BGK_SMAG_Q19 && k.scalar == LBM_SCALAR_Q6)
        return launch_face_storage<19, 6>(kp, k.storage, face, pack, f, phi, buf, st);
    if (k.model == LBM_CUMULANT_Q27 && k.scalar == LBM_SCALAR_Q7)
        return launch_face_storage<27, 7>(kp, k.storage, face, pack, f, phi, buf, st);
    if (k.model == LBM_CUMULANT_Q27 && k.scalar == LBM_SCALAR_Q27)
        return launch_face_storage<27, 27>(kp, k.storage, face, pack, f, phi, buf, st);
    return cudaErrorInvalidValue;
}

}  // namespace lbmgpu
