// lbm_staged.cu -- the fused AA stream + collide step with every population
// row segment moved between HBM and shared memory by the TMA engine
// (one-dimensional cp.async.bulk copies completing on mbarriers).
//
// Per node and step the arithmetic is that of the other step kernels
// (cumulant: lbm_cumulant_collide.cuh, Eq. 52-58 with the D3Q7 scalar,
// Eq. 27-30; BGK: lbm_bgk_collide.cuh, Eq. 17-35), the streaming that of the
// AA pattern described in lbm_common.cuh (Eq. 17).  What differs is how the
// bytes move.  A tile is a segment of TILE x-consecutive nodes of one
// (y, z) row (TILE = 1 KB of storage: 512 nodes in 16 bits, 256 in FP32),
// one node per thread.  For each population the tile reads one
// contiguous row segment and writes one: on even steps both are the tile's
// own x range; on odd steps the populations with c_x != 0 come from (go to)
// the range shifted by -c_x (+c_x), which is not 16-byte aligned, so the
// load takes the aligned window widened by 16 bytes on each side (clamped
// to the row) and the store takes its aligned interior, the few elements at
// its ragged ends being stored by their threads directly.
//
// Each block is persistent over tiles (grid = resident blocks of the whole
// GPU) and keeps NST stages of shared memory: while its warps collide tile
// i, the bulk loads of tiles i + 1 .. i + NST - 2 are in flight and the bulk
// stores of tile i - 1 drain.  The lanes of warp 0 issue the copies, one or
// two population rows each.  The bulk copy engine spends about the same
// time on a copy of 256 bytes as on one of 512 (measured: a 128-node tile
// moved FP32 rows at 5.7 TB/s and 16-bit rows at 3.2 TB/s, the same number
// of copies per second), so the tiles are sized for copies of 1 KB.  Waits
// on the mbarriers are bounded (LBM_DEVFLAG_TIMEOUT, then the block
// returns).
//
// In-place safety is that of the AA pattern: every element is read and
// written within a step by one node only, and that node's tile.  The widened
// load windows also read up to 16 bytes of the neighbouring tiles' rows,
// which those tiles may be rewriting; such elements are never used.
#include <algorithm>
#include <type_traits>

#include "lbm_bgk_collide.cuh"
#include "lbm_bulk.cuh"
#include "lbm_cumulant_collide.cuh"
#include "lbm_internal.h"

namespace lbmgpu {

namespace {

constexpr uint64_t WAIT_LIMIT_NS = 10000000000ull;   // 10 s: only a defect waits that long

// Bytes of one population row segment of a tile, and resident blocks per SM.
#ifndef LBM_STAGED_ROWBYTES
#define LBM_STAGED_ROWBYTES 512
#endif
#ifndef LBM_STAGED_BLOCKS
#define LBM_STAGED_BLOCKS 2
#endif

// (c + 1) of every D3Q27 direction packed two bits per direction, for lookups
// with a run-time direction index.
template <int A>
__host__ __device__ constexpr uint64_t pack_axis() {
    uint64_t v = 0;
    for (int d = 0; d < 27; ++d) {
        const int c = A == 0 ? cx27(d) : (A == 1 ? cy27(d) : cz27(d));
        v |= (uint64_t)(c + 1) << (2 * d);
    }
    return v;
}
__device__ __forceinline__ int c_of(uint64_t packed, int d) {
    return (int)((packed >> (2 * d)) & 3u) - 1;
}

// Shared-memory geometry of one stage: one slot per population row, each
// holding TX + 2 HALO elements (the tile's range widened by 16 bytes on both
// sides); with 16-bit storage the FP32 rest row of the scalar takes a slot
// of TX floats at the end.  TX: nodes per tile = threads per block.
template <int Q, int SL, typename S>
struct Geom {
    static constexpr int TX = LBM_STAGED_ROWBYTES / (int)sizeof(S);
    static constexpr int NS = ScalarLat<SL>::NS;
    static constexpr int D0 = ScalarLat<SL>::D0;
    static constexpr bool R32 = rest32<S, SL>();
    static constexpr int ES = sizeof(S);
    static constexpr int HALO = 16 / ES;
    static constexpr int SLOT = (TX + 2 * HALO) * ES;
    static constexpr int NSLOT = Q + NS;
    static constexpr int RAW = R32 ? (NSLOT - 1) * SLOT + TX * 4 : NSLOT * SLOT;
    static constexpr int BYTES = (RAW + 127) / 128 * 128;
    __host__ __device__ static constexpr int off(int j) {
        return (R32 && j == Q) ? (NSLOT - 1) * SLOT : ((R32 && j > Q) ? (j - 1) * SLOT : j * SLOT);
    }
};

template <typename S>
__device__ __forceinline__ float lds(const unsigned char* p) {
    if constexpr (std::is_same<S, float>::value) return *reinterpret_cast<const float*>(p);
    else if constexpr (std::is_same<S, __half>::value)
        return __half2float(*reinterpret_cast<const __half*>(p));
    else return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
}
template <typename S>
__device__ __forceinline__ void sts(unsigned char* p, float v) {
    if constexpr (std::is_same<S, float>::value) *reinterpret_cast<float*>(p) = v;
    else if constexpr (std::is_same<S, __half>::value)
        *reinterpret_cast<__half*>(p) = __float2half_rn(v);
    else *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16_rn(v);
}

// The collisions, on populations in storage units.
struct CumulantCollide {
    template <int SL, typename S>
    static __device__ __forceinline__ void run(const KParams& kp, float (&f)[27],
                                               float (&p)[ScalarLat<SL>::NS]) {
        constexpr bool s16 = !std::is_same<S, float>::value;
        constexpr bool fold = s16 && SL == 7;   // the collision applies the scales
        if constexpr (s16 && !fold) {
#pragma unroll
            for (int i = 0; i < 27; ++i) f[i] *= kp.isf;
#pragma unroll
            for (int k = 0; k < ScalarLat<SL>::NS; ++k) p[k] *= kp.isp;
        }
        collide_cumulant<SL, fold>(kp, f, p);
        if constexpr (s16 && !fold) {
#pragma unroll
            for (int i = 0; i < 27; ++i) f[i] *= kp.sf;
#pragma unroll
            for (int k = 0; k < ScalarLat<SL>::NS; ++k) p[k] *= kp.sp;
        }
    }
};
struct BgkCollide {
    template <int SL, typename S>
    static __device__ __forceinline__ void run(const KParams& kp, float (&f)[19],
                                               float (&p)[ScalarLat<SL>::NS]) {
        collide_bgk<!std::is_same<S, float>::value, SL>(kp, f, p);
    }
};

// A tile: x0 (multiple of TX), y, z and its node index at x0.
struct Tile {
    int x0, y, z;
    unsigned nb;
};
template <int TX>
__device__ __forceinline__ Tile tile_at(const KParams& kp, unsigned tile, int nxb) {
    Tile T;
    const unsigned r = tile / (unsigned)nxb;
    T.x0 = (int)(tile - r * (unsigned)nxb) * TX;
    T.y = (int)(r % (unsigned)kp.ny);
    T.z = (int)(r / (unsigned)kp.ny);
    T.nb = (unsigned)T.z * kp.nxny + (unsigned)T.y * kp.nx + (unsigned)T.x0;
    return T;
}

// Node index of the row (y + dy, z + dz) at x = 0, y periodic, z periodic or
// walled; false when z + dz lies beyond a wall.
__device__ __forceinline__ bool row_at(const KParams& kp, bool pz, int y, int z, int dy, int dz,
                                       unsigned& nb) {
    int yy = y + dy, zz = z + dz;
    yy = yy < 0 ? yy + kp.ny : (yy >= kp.ny ? yy - kp.ny : yy);
    if (zz < 0 || zz >= kp.nz) {
        if (!pz) return false;
        zz = zz < 0 ? zz + kp.nz : zz - kp.nz;
    }
    nb = (unsigned)zz * kp.nxny + (unsigned)yy * kp.nx;
    return true;
}

// Slot j of the population arrays: direction (D3Q27 order), its row and the
// row of the opposite direction in its array.
template <int Q, int D0>
struct SlotDir {
    int dir, row, orow;
    bool fluid;
    __device__ __forceinline__ SlotDir(int j) {
        fluid = j < Q;
        dir = fluid ? j : j - Q + D0;
        row = fluid ? j : j - Q;
        const int o = dir == 0 ? 0 : ((dir & 1) ? dir + 1 : dir - 1);
        orow = fluid ? o : o - D0;
    }
};

}  // namespace

// Gather (a1) of one node of a tile from the input stage `in`, except the
// populations whose upwind node lies across the x ends (bounce-back or
// periodic wrap, read from global memory).  GEN: the tile touches the x ends
// or a z wall; otherwise every source row is inside the box and no
// population needs a test.
template <int Q, int SL, typename S, bool ODD, bool GEN>
__device__ __forceinline__ void stage_gather(const KParams& kp, const Tile& T, int t,
                                             const S* __restrict__ f, const S* __restrict__ phi,
                                             const unsigned char* in, const unsigned (&zr)[3],
                                             const unsigned (&yr)[3], float (&fv)[Q],
                                             float (&pv)[ScalarLat<SL>::NS]) {
    using G = Geom<Q, SL, S>;
    constexpr int D0 = G::D0, HALO = G::HALO, ES = G::ES;
    const int nx = kp.nx, x = T.x0 + t;
    const unsigned N = kp.N;
    const bool px = (kp.flags & LBM_FLAG_PERIODIC_X) != 0;
    const bool pz = (kp.flags & LBM_FLAG_PERIODIC_Z) != 0;
    const bool zlo = !pz && T.z == 0, zhi = !pz && T.z == kp.nz - 1;
#pragma unroll
    for (int j = 0; j < G::NSLOT; ++j) {
        const int dir = j < Q ? j : j - Q + D0;
        const int row = j < Q ? j : j - Q;
        const int orow = j < Q ? opp(dir) : opp(dir) - D0;
        const S* arr = j < Q ? f : phi;
        const unsigned char* slot = in + G::off(j);
        float v;
        if (G::R32 && j == Q) {
            v = reinterpret_cast<const float*>(slot)[t];
        } else if (!ODD || dir == 0 || cx27(dir) == 0) {
            v = lds<S>(slot + (HALO + t) * ES);
        } else if (!GEN) {
            v = lds<S>(slot + (HALO - cx27(dir) + t) * ES);
        } else {
            const int cx = cx27(dir), cy = cy27(dir), cz = cz27(dir);
            const bool zin = !((cz > 0 && zlo) || (cz < 0 && zhi));
            const int xs = x - cx;
            if (!zin) {
                v = lds<S>(slot + (HALO + t) * ES);           // z wall: own slot, loaded
            } else if (xs < 0 || xs >= nx) {
                const unsigned g = px ? (unsigned)orow * N + zr[1 - cz] + yr[1 - cy] +
                                            (unsigned)(xs < 0 ? xs + nx : xs - nx)
                                      : (unsigned)row * N + zr[1] + yr[1] + (unsigned)x;
                v = LBM_IN(kp, LBM_SITE_STAGED, arr, arr + g, 1, (size_t)(j < Q ? Q : G::NS) * N)
                        ? Store<S>::ld(arr + g)
                        : 0.0f;
            } else {
                v = lds<S>(slot + (HALO - cx + t) * ES);
            }
        }
        if (j < Q) fv[j] = v;
        else pv[j - Q] = v;
    }
}

// Scatter (a6) of one node into the output stage `out`, except the ragged
// ends of the shifted rows and populations leaving across the x ends, which
// the thread stores to global memory itself.
template <int Q, int SL, typename S, bool ODD, bool GEN>
__device__ __forceinline__ void stage_scatter(const KParams& kp, const Tile& T, int t,
                                              S* __restrict__ f, S* __restrict__ phi,
                                              unsigned char* out, const unsigned (&zr)[3],
                                              const unsigned (&yr)[3], const float (&fv)[Q],
                                              const float (&pv)[ScalarLat<SL>::NS]) {
    using G = Geom<Q, SL, S>;
    constexpr int D0 = G::D0, HALO = G::HALO, ES = G::ES, TX = G::TX;
    const int nx = kp.nx, x = T.x0 + t;
    const unsigned N = kp.N;
    const bool px = (kp.flags & LBM_FLAG_PERIODIC_X) != 0;
    const bool pz = (kp.flags & LBM_FLAG_PERIODIC_Z) != 0;
    const bool zlo = !pz && T.z == 0, zhi = !pz && T.z == kp.nz - 1;
    // threads whose element of a row shifted by +1 (-1) falls outside the
    // aligned interior that the bulk store writes
    const bool rp = t < HALO - 1 || t == TX - 1, rm = t == 0 || t > TX - HALO;
#pragma unroll
    for (int j = 0; j < G::NSLOT; ++j) {
        const int dir = j < Q ? j : j - Q + D0;
        const int row = j < Q ? j : j - Q;
        const int orow = j < Q ? opp(dir) : opp(dir) - D0;
        S* arr = j < Q ? f : phi;
        unsigned char* slot = out + G::off(j);
        const float v = j < Q ? fv[j] : pv[j - Q];
        if (G::R32 && j == Q) {
            reinterpret_cast<float*>(slot)[t] = v;
        } else if (!ODD || dir == 0 || cx27(dir) == 0) {
            sts<S>(slot + (HALO + t) * ES, v);
        } else {
            const int cx = cx27(dir), cy = cy27(dir), cz = cz27(dir);
            const int xt = x + cx;
            const bool zin = !GEN || !((cz > 0 && zhi) || (cz < 0 && zlo));
            if (!zin) {
                sts<S>(slot + (HALO + t) * ES, v);            // z wall: own slot of opp
            } else if (GEN && (xt < 0 || xt >= nx)) {
                const unsigned g = px ? (unsigned)row * N + zr[1 + cz] + yr[1 + cy] +
                                            (unsigned)(xt < 0 ? xt + nx : xt - nx)
                                      : (unsigned)orow * N + zr[1] + yr[1] + (unsigned)x;
                if (LBM_IN(kp, LBM_SITE_STAGED, arr, arr + g, 1, (size_t)(j < Q ? Q : G::NS) * N))
                    Store<S>::st(arr + g, v);
            } else if (cx > 0 ? rp : rm) {
                const unsigned g = (unsigned)row * N + zr[1 + cz] + yr[1 + cy] + (unsigned)xt;
                if (LBM_IN(kp, LBM_SITE_STAGED, arr, arr + g, 1, (size_t)(j < Q ? Q : G::NS) * N))
                    Store<S>::st(arr + g, v);
            } else {
                sts<S>(slot + (HALO + cx + t) * ES, v);
            }
        }
    }
}

// Warp-specialised persistent step kernel: TX consumer threads (one node
// each) and one producer warp.  The producer issues every bulk copy: loads
// of tile k into input stage k % NIN (completing on full), stores of tile j
// from output stage j % NOUT once the consumers have filled it (ready), and
// frees an output stage (out_free) once its stores have read it.  The
// consumers wait for a tile's inputs, gather, release the input stage
// (in_done), collide, wait for a free output stage, scatter and signal ready.
// No block-wide barrier is taken inside the tile loop.
template <int Q, int SL, typename S, bool ODD, int NIN, int NOUT, typename Model>
__global__ void __launch_bounds__(Geom<Q, SL, S>::TX + 32, LBM_STAGED_BLOCKS)
    staged_step_kernel(KParams kp, S* __restrict__ f, S* __restrict__ phi) {
    using G = Geom<Q, SL, S>;
    constexpr int NS = G::NS, D0 = G::D0, HALO = G::HALO, ES = G::ES, TX = G::TX;
    constexpr int LAG = NIN - 1;   // tiles the loads run ahead of the stores
    constexpr uint64_t PX = pack_axis<0>(), PY = pack_axis<1>(), PZ = pack_axis<2>();
    static_assert(NIN >= 2 && NOUT >= 2, "two stages at least on each side");

    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[NIN], in_done[NIN], ready[NOUT], out_free[NOUT];
    __shared__ int abort_flag;

    const int t = threadIdx.x, lane = t & 31;
    const bool producer = t >= TX;
    const int nx = kp.nx, nxb = kp.nx / TX;
    const unsigned N = kp.N;
    const unsigned ntiles = (unsigned)nxb * kp.ny * kp.nz;
    const bool pz = (kp.flags & LBM_FLAG_PERIODIC_Z) != 0;
    float* const rest = G::R32 ? rest_row(phi, NS, N) : nullptr;
    const unsigned nmine =
        blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0u;
    unsigned char* const in_base = smem;
    unsigned char* const out_base = smem + NIN * G::BYTES;

    // bulk copies need 16-byte aligned shared addresses (uniform per block)
    if (smem_addr(smem) & 15u) {
        if (t == 0) atomicOr(kp.devflags, LBM_DEVFLAG_TIMEOUT);
        return;
    }
    if (t == 0) {
        for (int s = 0; s < NIN; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&in_done[s], TX);
        }
        for (int s = 0; s < NOUT; ++s) {
            mbar_init(&ready[s], TX);
            mbar_init(&out_free[s], 1);
        }
        abort_flag = 0;
        mbar_fence_init();
    }
    __syncthreads();

    // the test hook of the failure path: a short limit, and each block's
    // first tile announced on its barrier but never copied (the phase never
    // completes, and no copy is in flight on it)
    const bool stall = (kp.flags & LBM_FLAG_TEST_STALL) != 0;
    const uint64_t limit = stall ? 100000000ull : WAIT_LIMIT_NS;

    // bounded wait that also gives up once another warp has given up
    auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
        if (mbar_try_wait(bar, parity)) return true;
        const uint64_t t0 = global_ns();
        while (!mbar_try_wait(bar, parity)) {
            if (*(volatile int*)&abort_flag) return false;
            if (global_ns() - t0 > limit) {
                atomicExch(&abort_flag, 1);
                return false;
            }
        }
        return true;
    };

    if (producer) {
        // lane l issues the copies of slots l and l + 32
        auto issue_loads = [&](unsigned k) {
            const int s = (int)(k % NIN);
            const Tile T = tile_at<TX>(kp, blockIdx.x + k * gridDim.x, nxb);
            unsigned char* sb = in_base + s * G::BYTES;
            const void* src[2];
            uint32_t dst[2], nbytes[2];
            uint32_t total = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                nbytes[h] = 0;
                if (j >= G::NSLOT) continue;
                const SlotDir<Q, D0> sd(j);
                const S* base = sd.fluid ? f : phi;
                uint32_t o = G::off(j);
                if (G::R32 && j == Q) {
                    src[h] = rest + T.nb;
                    dst[h] = o;
                    nbytes[h] = TX * 4;
                    if (!LBM_IN(kp, LBM_SITE_STAGED, rest, rest + T.nb, TX, N)) nbytes[h] = 0;
                } else {
                    const S* p = base + (size_t)sd.row * N + T.nb;   // own row segment
                    uint32_t bytes = TX * ES;
                    o += HALO * ES;
                    if (ODD && sd.dir != 0) {
                        const int cx = c_of(PX, sd.dir), cy = c_of(PY, sd.dir),
                                  cz = c_of(PZ, sd.dir);
                        unsigned nbs;
                        if (row_at(kp, pz, T.y, T.z, -cy, -cz, nbs)) {
                            const S* ob = base + (size_t)sd.orow * N + nbs;
                            if (cx == 0) {
                                p = ob + T.x0;
                            } else {
                                const int lo = max(T.x0 - HALO, 0),
                                          hi = min(T.x0 + TX + HALO, nx);
                                p = ob + lo;
                                o += (lo - T.x0) * ES;
                                bytes = (hi - lo) * ES;
                            }
                        }
                    }
                    src[h] = p;
                    dst[h] = o;
                    nbytes[h] = bytes;
                    if (!LBM_IN(kp, LBM_SITE_STAGED, base, p, bytes / ES,
                                (size_t)(sd.fluid ? Q : NS) * N))
                        nbytes[h] = 0;
                }
                total += nbytes[h];
            }
            total = __reduce_add_sync(0xffffffffu, total);
            if (lane == 0) mbar_arrive_expect_tx(&full[s], total);
            __syncwarp();
            if (stall && k == 0) return;
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (nbytes[h]) bulk_load(sb + dst[h], src[h], nbytes[h], &full[s]);
        };
        auto issue_stores = [&](unsigned jt) {
            const int o8 = (int)(jt % NOUT);
            const Tile T = tile_at<TX>(kp, blockIdx.x + jt * gridDim.x, nxb);
            const unsigned char* sb = out_base + o8 * G::BYTES;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int j = lane + 32 * h;
                if (j >= G::NSLOT) continue;
                const SlotDir<Q, D0> sd(j);
                S* base = sd.fluid ? f : phi;
                const uint32_t o = G::off(j);
                if (G::R32 && j == Q) {
                    if (LBM_IN(kp, LBM_SITE_STAGED, rest, rest + T.nb, TX, N))
                        bulk_store(rest + T.nb, sb + o, TX * 4);
                    continue;
                }
                void* p = base + (size_t)sd.orow * N + T.nb;     // own slot of the opposite
                uint32_t so = o + HALO * ES, bytes = TX * ES;
                if (ODD && sd.dir != 0) {
                    const int cx = c_of(PX, sd.dir), cy = c_of(PY, sd.dir), cz = c_of(PZ, sd.dir);
                    unsigned nbt;
                    if (row_at(kp, pz, T.y, T.z, cy, cz, nbt)) {
                        S* tb = base + (size_t)sd.row * N + nbt + T.x0;
                        if (cx == 0) {
                            p = tb;
                        } else if (cx > 0) {
                            p = tb + HALO;
                            so = o + 2 * HALO * ES;
                            bytes = (TX - HALO) * ES;
                        } else {
                            p = tb;
                            bytes = (TX - HALO) * ES;
                        }
                    }
                }
                if (LBM_IN(kp, LBM_SITE_STAGED, base, (S*)p, bytes / ES,
                           (size_t)(sd.fluid ? Q : NS) * N))
                    bulk_store(p, sb + so, bytes);
            }
            bulk_commit();
        };

        unsigned issued = 0;   // tiles whose loads were issued
        bool ok = true;
        for (unsigned k = 0; ok && k < nmine + LAG; ++k) {
            if (k < nmine) {
                if (k >= NIN) ok = wait(&in_done[k % NIN], ((k / NIN) - 1) & 1u);
                if (!ok) break;
                issue_loads(k);
                issued = k + 1;
            }
            if (k >= (unsigned)LAG) {
                const unsigned jt = k - LAG;
                ok = wait(&ready[jt % NOUT], (jt / NOUT) & 1u);
                if (!ok) break;
                issue_stores(jt);
                if (jt >= 1) {
                    bulk_wait_read<1>();   // the stores of tile jt - 1 have left their stage
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&out_free[(jt - 1) % NOUT]);
                }
            }
        }
        bulk_wait_all();
        if (!ok) {
            if (lane == 0) atomicOr(kp.devflags, LBM_DEVFLAG_TIMEOUT);
            // loads still in flight land in this block's shared memory: let
            // them complete (bounded) before the block exits
            for (unsigned k = issued > (unsigned)NIN ? issued - NIN : 0u; k < issued; ++k)
                mbar_wait_bounded(&full[k % NIN], (k / NIN) & 1u, limit);
        }
        return;
    }

    // consumers
    for (unsigned i = 0; i < nmine; ++i) {
        const int s = (int)(i % NIN), o8 = (int)(i % NOUT);
        const Tile T = tile_at<TX>(kp, blockIdx.x + i * gridDim.x, nxb);
        const unsigned zr[3] = {(unsigned)(T.z == 0 ? kp.nz - 1 : T.z - 1) * kp.nxny,
                                (unsigned)T.z * kp.nxny,
                                (unsigned)(T.z == kp.nz - 1 ? 0 : T.z + 1) * kp.nxny};
        const unsigned yr[3] = {(unsigned)(T.y == 0 ? kp.ny - 1 : T.y - 1) * kp.nx,
                                (unsigned)T.y * kp.nx,
                                (unsigned)(T.y == kp.ny - 1 ? 0 : T.y + 1) * kp.nx};
        const bool gen = ODD && (T.x0 == 0 || T.x0 + TX == nx ||
                                 (!pz && (T.z == 0 || T.z == kp.nz - 1)));
        if (!wait(&full[s], (i / NIN) & 1u)) break;
        const unsigned char* in = in_base + s * G::BYTES;
        float fv[Q], pv[NS];
        if (gen) stage_gather<Q, SL, S, ODD, true>(kp, T, t, f, phi, in, zr, yr, fv, pv);
        else stage_gather<Q, SL, S, ODD, false>(kp, T, t, f, phi, in, zr, yr, fv, pv);
        mbar_arrive(&in_done[s]);
        if (!(kp.flags & LBM_FLAG_NO_COLLIDE)) Model::template run<SL, S>(kp, fv, pv);
        if constexpr (G::R32) feed_rest<S>(pv);
        if (i >= (unsigned)NOUT && !wait(&out_free[o8], ((i / NOUT) - 1) & 1u)) break;
        unsigned char* out = out_base + o8 * G::BYTES;
        if (gen) stage_scatter<Q, SL, S, ODD, true>(kp, T, t, f, phi, out, zr, yr, fv, pv);
        else stage_scatter<Q, SL, S, ODD, false>(kp, T, t, f, phi, out, zr, yr, fv, pv);
        fence_proxy_async_smem();
        mbar_arrive(&ready[o8]);
    }
}

namespace {

template <int Q, int SL, typename S, bool ODD, typename Model>
cudaError_t launch_typed(const KParams& kp, S* f, S* phi, cudaStream_t st) {
    // one block per SM: TX consumer threads + one producer warp, three input
    // and two output stages of 37 KB (16-bit storage)
    constexpr int NIN = 3, NOUT = 2;
    using G = Geom<Q, SL, S>;
    auto kern = staged_step_kernel<Q, SL, S, ODD, NIN, NOUT, Model>;
    const size_t smem = (size_t)(NIN + NOUT) * G::BYTES;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    static int per_sm[64];   // resident blocks per SM, per device (0: not yet known)
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (per_sm[dev] == 0) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, G::TX + 32, smem);
        if (e != cudaSuccess) return e;
        per_sm[dev] = b > 0 ? b : 1;
    }
    int nsm = 0;
    e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    const long long ntiles = (long long)(kp.nx / G::TX) * kp.ny * kp.nz;
    const long long grid = std::min<long long>(ntiles, (long long)nsm * per_sm[dev]);
    kern<<<(unsigned)grid, G::TX + 32, smem, st>>>(kp, f, phi);
    return cudaGetLastError();
}

template <int Q, int SL, typename S, typename Model>
cudaError_t launch_parity(const KParams& kp, bool odd, void* f, void* phi, cudaStream_t st) {
    if (odd) return launch_typed<Q, SL, S, true, Model>(kp, (S*)f, (S*)phi, st);
    return launch_typed<Q, SL, S, false, Model>(kp, (S*)f, (S*)phi, st);
}

}  // namespace

bool staged_step_applies(const KParams& kp, Kind k) {
    // opt-in; 16-bit storage, tiles of LBM_STAGED_ROWBYTES / 2 nodes
    if (!(kp.flags & LBM_FLAG_TMA_STAGED) || (kp.flags & LBM_FLAG_ONE_NODE) || !kp.devflags ||
        kp.wide)
        return false;
    if (k.storage == LBM_FP32 || kp.nx % (LBM_STAGED_ROWBYTES / 2) != 0) return false;
    return k.model == LBM_CUMULANT_Q27 && k.scalar == LBM_SCALAR_Q7;
}

cudaError_t launch_staged_step(const KParams& kp, Kind k, bool odd, void* f, void* phi,
                               cudaStream_t st) {
    if (k.model == LBM_CUMULANT_Q27 && k.scalar == LBM_SCALAR_Q7) {
        switch (k.storage) {
            case LBM_FP16S: return launch_parity<27, 7, __half, CumulantCollide>(kp, odd, f, phi, st);
            case LBM_BF16S:
                return launch_parity<27, 7, __nv_bfloat16, CumulantCollide>(kp, odd, f, phi, st);
        }
    }
    return cudaErrorInvalidValue;
}

}  // namespace lbmgpu
