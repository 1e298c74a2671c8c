// One Wicker-Skamarock RK3 stage, fused (Sec. 1.1 "ASUCA on GPU"):
//   phi = (rho phi) / rho                     (one reciprocal of rho per cell)
//   face values by the Koren limiter in i, j, k, upwind by sign(M)
//   R = -[dX/dx + dY/dy + dZ/dz] + tendency,  Y_out = Y_base + cdt R
//
// Mapping: a CTA owns a 32 x TY tile of (i, j) columns, one warp per row, and
// marches k (parallel in I/J, sequential in K; Sec. 1.1, Sec. 1.2): upward, or
// downward for the third stage that carries the top-down column pass.
// Level planes of the stage input stream through a ring of D shared-memory
// slots, each holding every field of the tile plus a halo of 4 columns in i
// (the TMA box must start on a 16-byte boundary; 2 are used) and 2 rows in j:
//   * from the library's padded stage buffers, one 4D TMA box per level
//     (cp.async.bulk.tensor, completion on an mbarrier).  The stage that
//     produced the buffer wrote phi (not rho*phi) and the periodic halo
//     ghosts, so the level is used as it lands;
//   * from the caller's unpadded fields (rho*phi): for tiles whose halo lies
//     inside the domain, three TMA boxes per level (rho, rho*theta, the N
//     tracers); at the periodic edges, per-thread cp.async copies with the
//     wrap done in the index arithmetic.  These levels are converted in place
//     to phi, once per cell.
// Levels are requested D-2 levels ahead.  Every face is reconstructed once:
// i+1/2 by each thread (the i-1/2 flux comes from the neighbouring lane by
// shuffle), j+1/2 by each thread into shared memory, the vertical face ahead of
// the march by each thread with the one behind carried in registers; the faces
// on the tile's left and
// bottom edges are computed by warps dealt round-robin.  A face's upwind,
// downwind and far cells are picked by address from the sign of M, so the
// limiter arithmetic has no per-field selects.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <type_traits>

#include "common.cuh"
#include "smem_attr.cuh"

namespace asuca {

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the mbarrier phase with the given parity; gives up after about one
// second of wall time and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const uint32_t addr = smem_u32(bar);
    uint64_t t0 = 0;
    for (uint32_t it = 0;; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
        if (it == 0) t0 = global_ns();
        else if ((it & 63u) == 0 && global_ns() - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int x, int y, int z, int w,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_u32(dst)), "l"(src), "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ------------------------------------------------------------------ the kernel

// One tile of one stage: the CTA computes columns [i0, i0+32) x [j0, j0+TY)
// for every level.  Returns true when a level's data did not arrive within the
// wait limit (the status word has been set).  The caller's CTA owns smem_raw;
// the function begins and ends with a CTA-wide barrier, so consecutive tiles
// may reuse the same shared memory and mbarriers.
// The default output of a tile: the stage result is written to p.yout.
struct NoHook {
    static constexpr bool active = false, keep_output = true, own_rho = false, defers = false;
    template <typename T, int NF>
    __device__ __forceinline__ void level(int, const T (&)[NF], bool, T, T) {}
    __device__ __forceinline__ void early() {}
    __device__ __forceinline__ void done(bool) {}
};

// Slot layouts of the ring (StageShape): the caller's fields (stage 1) land
// as planes, the library's padded stage buffers as phi pairs.
constexpr int LAYOUT_RAW = 0, LAYOUT_PAIR = 1;

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float2; };
template <> struct Vec2<double> { using type = double2; };

// DOWN marches the levels from the top down (the ring, the faces and the
// carried flux all run in march order; level k = nz - 1 - t at march step t),
// which gives the same arithmetic per cell, so the result is bit-identical to
// the upward march.  An active Hook takes each level's result, instead
// of the writes to p.yout unless it has keep_output: hook.level(k, out, valid,
// rho_next, rho_h), where rho_next is the density result of the next level of
// the march (the same expression that level will evaluate); a hook with
// own_rho receives in rho_h and rho_next the density Y^n + hcdt R instead of
// the stage's (the same expression with p.hcdt for cdt).  hook.early() runs
// before each level's faces (a hook may defer a level's work to it, so that
// the work interleaves with the next level's faces), hook.done(valid) after
// the last level.
// The fields are processed in pairs (1, 2), (3, 4), ...: a pair shares every
// operation of its face reconstruction and divergence (packed FP32x2 for
// float), and with the pair layout its operands arrive in one load.
template <typename T, int NF, int LIM, bool REC, int TYV, bool DOWN, typename Hook, int LAY>
__device__ __forceinline__ bool stage_tile_h(const StageParams<T> &p, const CUtensorMap *tmap, int i0, int j0,
                                             unsigned char *smem_raw, Hook &hook,
                                             const CUtensorMap *umaps = nullptr) {
    // the tensor maps of the caller's fields: p.umap, or a copy in global
    // memory when p itself lies in shared memory (TMA reads no map from there)
    const CUtensorMap *um = umaps ? umaps : p.umap;
    static_assert(!(DOWN && REC), "branch recording marches upward");
    using S = StageShape<T, NF, TYV>;
    using T2 = typename Vec2<T>::type;
    constexpr int TX = S::TX, TY = S::TY, D = S::D, SX = S::SX, SY = S::SY, NT = S::NT, NPF = S::NPF;
    constexpr int NTHR = TX * TY;
    constexpr int FE = SY * SX;                   // raw layout: elements of one field in a slot
    constexpr bool PAIRL = LAY == LAYOUT_PAIR;
    // a slot cell (sy, sx): raw field f at f FE + sy SX + sx; pair layout pair q
    // at (sy NPF + q) 2 SX + 2 sx (two values)
    constexpr int XS = PAIRL ? 2 : 1;             // one cell along i
    constexpr int YS = PAIRL ? 2 * NPF * SX : SX; // one row
    constexpr int QS = 2 * SX;                    // one pair (pair layout)
    // The slot cells the stencil reads (no corners), dealt to the threads in
    // pairs of neighbours along i for the copies and the conversion to phi
    // (raw layout only): TY rows of TX + 4 cells (i0-2 .. i0+TX+1) and 4 halo
    // rows of TX cells.
    constexpr int PR = (TX + 4) / 2, PH = TX / 2;
    constexpr int NPAIR = TY * PR + 4 * PH;
    constexpr int MAXC = PAIRL ? 1 : (NPAIR + NTHR - 1) / NTHR;
    static_assert((FE * sizeof(T)) % 128 == 0, "each field of a slot must start on a 128-byte boundary");
    constexpr bool PACK = std::is_same<T, float>::value;

    T *ring = reinterpret_cast<T *>(smem_raw);
    T2 *ysm = reinterpret_cast<T2 *>(smem_raw + S::RING_BYTES);               // [NPF][TY+1][TX]
    T2 *xbs = reinterpret_cast<T2 *>(smem_raw + S::RING_BYTES + S::YS_BYTES); // [NPF][TY]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw + S::RING_BYTES + S::YS_BYTES + S::XB_BYTES);

    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TX + tx;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    // element offsets within a field fit in 32 bits (the host checks), which
    // keeps the per-field address arithmetic to one 32-bit index
    const unsigned plane = (unsigned)p.plane;
    const int i = i0 + tx, j = j0 + ty;
    const bool valid = (i < nx) && (j < ny);
    const bool open = p.open != 0;
    // threads past the domain's edge compute nothing they keep: periodic tiles
    // wrap their indices, open ones clamp them (nothing lies beyond the edge)
    const int ic = open ? min(i, nx - 1) : wrap_index(i, nx), jc = open ? min(j, ny - 1) : wrap_index(j, ny);
    const unsigned own = (unsigned)(jc * nx + ic);
    // mass-flux indices: periodic, mu and mv share the cell's index (faces
    // i+1/2, j+1/2) and the faces i-1/2, j-1/2 wrap; open, face i-1/2 of cell i
    // is mu[j][i] of a row of nx+1 faces and face j-1/2 is mv[j][i]
    const unsigned u_own = open ? (unsigned)(jc * (nx + 1) + ic + 1) : own;
    const unsigned u_left = open ? (unsigned)(jc * (nx + 1) + ic) : (unsigned)(jc * nx + wrap_index(ic - 1, nx));
    const unsigned v_own = open ? (unsigned)((jc + 1) * nx + ic) : own;
    const unsigned v_down = open ? own : (unsigned)(wrap_index(jc - 1, ny) * nx + ic);
    const unsigned plane_u = (unsigned)p.plane_u, plane_v = (unsigned)p.plane_v;
    // Input paths: a padded stage buffer (phi pairs, one 4D TMA box per level);
    // the caller's fields (rho*phi) by TMA when the tile's halo lies inside the
    // domain, else by per-thread cp.async with the periodic wrap.
    constexpr bool pad_in = PAIRL;   // the pair layout is the padded input's (always so for open boundaries)
    const bool user_tma = !pad_in && p.user_tma && i0 >= 4 && i0 + TX + 4 <= nx && j0 >= 2 && j0 + TY + 2 <= ny;
    const bool tma = pad_in || user_tma;
    constexpr bool conv = !pad_in;

    __syncthreads();   // the previous tile (if any) is done with the shared memory
    if (tma && tid == 0) {
        for (int s = 0; s < D; s++) mbar_init(&bars[s], 1);
        fence_proxy_async();
    }

    // slot cell pairs (sx even, so a pair is one aligned 2-element vector)
    // this thread copies (cp.async path) and converts (raw layout)
    int soff[MAXC];
    unsigned goff[MAXC], goff1[MAXC];
    int nc = 0;
#pragma unroll
    for (int q = 0; q < MAXC; q++) {
        const int c = tid + q * NTHR;
        soff[q] = 0;
        goff[q] = goff1[q] = 0;
        if (!PAIRL && c < NPAIR) {
            int sy, sx;
            if (c < TY * PR) {
                sy = 2 + c / PR;
                sx = 2 + 2 * (c % PR);
            } else {
                const int c2 = c - TY * PR;
                const int r = c2 / PH;
                sx = 4 + 2 * (c2 % PH);
                sy = r < 2 ? r : TY + r;
            }
            soff[q] = sy * SX + sx;   // sx even
            const int gj = wrap_index(j0 + sy - 2, ny) * nx;
            goff[q] = (unsigned)(gj + wrap_index(i0 + sx - 4, nx));
            goff1[q] = (unsigned)(gj + wrap_index(i0 + sx - 3, nx));
            nc = q + 1;
        }
    }
    __syncthreads();

    // every field of the caller's input aligned to a pair of elements (the
    // cp.async path then copies adjacent cell pairs in one request)
    bool yin_pairs = true;
#pragma unroll
    for (int f = 0; f < NF; f++) yin_pairs = yin_pairs && (reinterpret_cast<uintptr_t>(p.yin[f]) % (2 * sizeof(T))) == 0;

    // ring slots of march steps t-1 .. t+2 and of the request t+D-2, rotated
    // by one slot per step (slot(n) = ring + (n mod D) SLOT_ELEMS)
    auto slot = [&](int lev) -> T * { return ring + (size_t)(lev % D) * S::SLOT_ELEMS; };

    int issued = 0, seen = 0;   // TMA levels [0, issued) requested, [0, seen) seen complete
    auto level_of = [&](int t) { return DOWN ? nz - 1 - t : t; };
    auto issue = [&](int t) {
        const int lev = level_of(t);
        if (tma) {
            if (t < nz) {
                issued = t + 1;
                if (tid == 0) {
                    uint64_t *bar = &bars[t % D];
                    T *dst = slot(t);
                    if (pad_in) {
                        // the phi pairs: the map's dimensions are (2 pitch, pairs, rows, levels)
                        mbar_expect_tx(bar, S::TX_BYTES_PAIR);
                        tma_load_4d(dst, tmap, 2 * i0, 0, j0, lev, bar);
                    } else {
                        mbar_expect_tx(bar, S::TX_BYTES);
                        tma_load_3d(dst, um + 0, i0 - 4, j0 - 2, lev, bar);
                        tma_load_3d(dst + FE, um + 1, i0 - 4, j0 - 2, lev, bar);
                        if (NF > 2) tma_load_4d(dst + 2 * FE, um + 2, i0 - 4, j0 - 2, lev, 0, bar);
                    }
                }
            }
        } else {
            if (t < nz) {
                T *sl = slot(t);
                const unsigned lb = (unsigned)lev * plane;
#pragma unroll
                for (int q = 0; q < MAXC; q++) {
                    if (q < nc) {
                        unsigned g0 = lb + goff[q], g1 = lb + goff1[q];
                        int s0 = soff[q];
                        ASUCA_BC(g0, (long long)nz * plane, p.status);
                        ASUCA_BC(g1, (long long)nz * plane, p.status);
                        ASUCA_BC(s0, S::SLOT_ELEMS - (NF - 1) * FE - 1, p.status);
                        // the pair's two cells adjacent and aligned in every field:
                        // one copy of both (s0 is even, so the slot side is aligned)
                        if (yin_pairs && g1 == g0 + 1 && !(g0 & 1u)) {
#pragma unroll
                            for (int f = 0; f < NF; f++) cp_async<2 * sizeof(T)>(sl + f * FE + s0, p.yin[f] + g0);
                        } else {
#pragma unroll
                            for (int f = 0; f < NF; f++) {
                                cp_async<sizeof(T)>(sl + f * FE + s0, p.yin[f] + g0);
                                cp_async<sizeof(T)>(sl + f * FE + s0 + 1, p.yin[f] + g1);
                            }
                        }
                    }
                }
            }
            cp_async_commit();
        }
    };

    // convert the cell pairs this thread owns in the slot of level lev from
    // rho*phi to phi (one reciprocal of rho per cell, one vector multiply per field)
    auto convert = [&](int lev) {
        T *sl = slot(lev);
#pragma unroll
        for (int q = 0; q < MAXC; q++) {
            if (q < nc) {
                const T2 rho = *reinterpret_cast<const T2 *>(sl + soff[q]);
                const T r0 = recip(rho.x), r1 = recip(rho.y);
#pragma unroll
                for (int f = 1; f < NF; f++) {
                    T2 *v = reinterpret_cast<T2 *>(sl + f * FE + soff[q]);
                    T2 w = *v;
                    if constexpr (PACK) {
                        w = __fmul2_rn(w, make_float2(r0, r1));
                    } else {
                        w.x *= r0;
                        w.y *= r1;
                    }
                    *v = w;
                }
            }
        }
    };
    // wait for level lev to land (TMA) and convert it if it holds rho*phi
    auto arrive = [&](int lev) -> bool {
        if (!mbar_wait(&bars[lev % D], (lev / D) & 1)) return false;
        seen = lev + 1;
        if (conv) convert(lev);
        return true;
    };

    // the two values of pair q at offset off of a slot (raw layout: fields
    // 2q+1 and 2q+2, the second 0 past the last field)
    auto ld2 = [&](const T *sl, int q, int off) -> T2 {
        if constexpr (PAIRL) {
            int e = q * QS + off;
            ASUCA_BC(e, S::SLOT_ELEMS - 1, p.status);
            return *reinterpret_cast<const T2 *>(sl + e);
        } else {
            // fields 2q+1 and (when it exists) 2q+2 of the slot at off
            ASUCA_BC(off, S::SLOT_ELEMS - (2 * q + 2 <= NT ? 2 * q + 2 : 2 * q + 1) * FE, p.status);
            T2 v;
            v.x = sl[(2 * q + 1) * FE + off];
            v.y = (2 * q + 2 <= NT) ? sl[(2 * q + 2) * FE + off] : T(0);
            return v;
        }
    };

    bool timed_out = false;
    // ---- prologue: request levels 0 .. D-3, make levels 0 and 1 ready
#pragma unroll 1
    for (int lev = 0; lev <= D - 3; lev++) issue(lev);
    if (tma) {
        if (!arrive(0)) timed_out = true;
        else if (nz > 1 && !arrive(1)) timed_out = true;
    } else {
        cp_async_wait<D - 3>();
        convert(0);
        cp_async_wait<D - 4>();
        if (nz > 1) convert(1);
    }

    const T cdt = p.cdt;
    const T ax = -cdt * p.rdx, ay = -cdt * p.rdy;   // out = base + ax dX + ay dY + az dZ + cdt t
    const int warp = ty, lane = tx;
    const int er = lane % TY;   // the tile row whose i0-1/2 faces this lane computes
    // MV through face j0-1/2 of column ic, MU through face i0-1/2 of row er
    const unsigned edge_b = open ? (unsigned)(j0 * nx + ic) : (unsigned)(wrap_index(j0 - 1, ny) * nx + ic);
    const unsigned edge_l = open ? (unsigned)(min(j0 + er, ny - 1) * (nx + 1) + i0)
                                 : (unsigned)(wrap_index(j0 + er, ny) * nx + wrap_index(i0 - 1, nx));
    // tiles that hold cells whose values are also periodic ghosts of the padded output
    const bool ghost_x = !open && ((i0 < 2) || (i0 + TX > nx - 2));
    const bool ghost_y = !open && ((j0 < 2) || (j0 + TY > ny - 2));

    T zlo0 = T(0);    // the density's flux through the face behind the march (M itself)
    T2 zlo[NPF];      // the pairs' fluxes through that face
#pragma unroll
    for (int q = 0; q < NPF; q++) zlo[q].x = zlo[q].y = T(0);

    // per-level mass fluxes, requested one level ahead (the faces need them first)
    // mwp is the flux through the face the march reaches next: k+1/2 upward
    // (mw[k + 1]), k-1/2 downward (mw[k]); zero at the lid
    T mup, mum, mvp, mvm, mwp, meb, mel;
    T nmup, nmum, nmvp, nmvm, nmwp, nmeb, nmel, nrho;
    auto prefetch = [&](int k) {
        const unsigned kb = (unsigned)k * plane, kbu = (unsigned)k * plane_u, kbv = (unsigned)k * plane_v;
        unsigned a_up = kbu + u_own, a_ul = kbu + u_left, a_vp = kbv + v_own, a_vd = kbv + v_down,
                 a_w = DOWN ? kb + own : kb + plane + own, a_eb = kbv + edge_b, a_el = kbu + edge_l, a_r = kb + own;
        ASUCA_BC(a_up, (long long)nz * plane_u, p.status);
        ASUCA_BC(a_ul, (long long)nz * plane_u, p.status);
        ASUCA_BC(a_el, (long long)nz * plane_u, p.status);
        ASUCA_BC(a_vp, (long long)nz * plane_v, p.status);
        ASUCA_BC(a_vd, (long long)nz * plane_v, p.status);
        ASUCA_BC(a_eb, (long long)nz * plane_v, p.status);
        ASUCA_BC(a_w, (long long)(nz + 1) * plane, p.status);
        ASUCA_BC(a_r, (long long)nz * plane, p.status);
        nmup = p.mu[a_up];
        nmum = p.mu[a_ul];
        nmvp = p.mv[a_vp];
        nmvm = p.mv[a_vd];
        if (DOWN) nmwp = (k > 0) ? p.mw[a_w] : T(0);
        else nmwp = (k < nz - 1) ? p.mw[a_w] : T(0);
        nmeb = p.mv[a_eb];
        nmel = p.mu[a_el];
        if (Hook::active) nrho = p.ybase[0][a_r];
    };
    auto advance = [&]() {
        mup = nmup; mum = nmum; mvp = nmvp; mvm = nmvm; mwp = nmwp; meb = nmeb; mel = nmel;
    };
    prefetch(level_of(0));
    advance();

    const int cy = ty + 2, cx = tx + 4, cc = cy * YS + cx * XS;
    // padded output (pair layout): the cell's element offset, and the pair stride
    const long long q2 = 2 * p.opitch;
    const bool has_tend = p.tend != nullptr;

    // the flux of pair q through a face from its upwind cell c, downwind cell
    // o and far upwind cell f; one field only for the last pair of an odd count
    auto flux2 = [&](int q, T2 c, T2 o, T2 f, T m) -> T2 {
        T2 r;
        if constexpr (PACK) {
            if (2 * q + 2 <= NT) return face_flux2<LIM>(c, o, f, m);
        }
        r.x = face_flux<LIM>(c.x, o.x, f.x, m);
        r.y = (2 * q + 2 <= NT) ? face_flux<LIM>(c.y, o.y, f.y, m) : T(0);
        return r;
    };

#pragma unroll 1
    for (int t = 0; t < nz; t++) {
        const int k = level_of(t);
        // ---- march step t+2 must be resident (and hold phi) before anyone computes step t
        if (t + 2 < nz) {
            if (tma) {
                if (!arrive(t + 2)) timed_out = true;
            } else {
                cp_async_wait<(D >= 5 ? D - 5 : 0)>();
                convert(t + 2);
            }
        }
        if (tma) fence_proxy_async();
        if (__syncthreads_or(timed_out)) {
            timed_out = true;
            break;
        }
        issue(t + D - 2);   // into the slot of march step t-2, which nobody reads any more
        // Y^n of this level: used after the faces, which cover the load latency
        T yb0;
        T2 yb[NPF];
        {
            unsigned kb = (unsigned)k * plane + own;
            ASUCA_BC(kb, (long long)nz * plane, p.status);
            yb0 = p.ybase[0][kb];
#pragma unroll
            for (int q = 0; q < NPF; q++) {
                yb[q].x = p.ybase[2 * q + 1][kb];
                yb[q].y = (2 * q + 2 <= NT) ? p.ybase[2 * q + 2][kb] : T(0);
            }
        }
        if (t + 1 < nz) prefetch(level_of(t + 1));
        if constexpr (Hook::defers) hook.early();   // a hook's work left from the previous level, beside these faces

        // ---- faces: upwind cell c, downwind cell o and far upwind cell by address
        // march steps t-1 .. t+2 (ghost levels copy the boundary cell)
        const T *Sk = slot(t);
        const T *Skm = slot(t > 0 ? t - 1 : 0);
        const T *Skp = slot(t + 1 < nz ? t + 1 : nz - 1);
        const T *Skp2 = slot(t + 2 < nz ? t + 2 : nz - 1);
        const bool top = (t == nz - 1);   // no face ahead of the last step
        // upwind cell of the face ahead: step t when the flux points along the
        // march (upward march: M >= 0; downward: M < 0, since M = 0 counts as upward)
        const bool ux = mup >= T(0), uy = mvp >= T(0), uz = DOWN ? (mwp < T(0)) : (mwp >= T(0));
        const int xc = cc + (ux ? 0 : XS), xo = cc + (ux ? XS : 0), xf = cc + (ux ? -XS : 2 * XS);
        const int yc = cc + (uy ? 0 : YS), yo = cc + (uy ? YS : 0), yf = cc + (uy ? -YS : 2 * YS);
        const T *zc = (uz ? Sk : Skp) + cc, *zo = (uz ? Skp : Sk) + cc, *zf = (uz ? Skm : Skp2) + cc;
        T2 xp[NPF], yp[NPF], zp[NPF];
#pragma unroll
        for (int q = 0; q < NPF; q++) {
            const T2 cxv = ld2(Sk, q, xc), oxv = ld2(Sk, q, xo), fxv = ld2(Sk, q, xf);
            const T2 cyv = ld2(Sk, q, yc), oyv = ld2(Sk, q, yo), fyv = ld2(Sk, q, yf);
            T2 czv, ozv, fzv;
            if (!top) {
                czv = ld2(zc, q, 0);
                ozv = ld2(zo, q, 0);
                fzv = ld2(zf, q, 0);
            }
            if constexpr (REC) {
                // the adjoint's record: each face's value and limiter branch
                int2 bx, by, bz = make_int2(0, 0);
                T2 vx, vy, vz;
                if constexpr (PACK) {
                    vx = face_val2_br<LIM>(cxv, oxv, fxv, bx);
                    vy = face_val2_br<LIM>(cyv, oyv, fyv, by);
                    if (!top) vz = face_val2_br<LIM>(czv, ozv, fzv, bz);
                    else vz = make_float2(0.f, 0.f);
                } else {
                    vx.x = face_val_br<LIM>(cxv.x, oxv.x, fxv.x, bx.x);
                    vx.y = face_val_br<LIM>(cxv.y, oxv.y, fxv.y, bx.y);
                    vy.x = face_val_br<LIM>(cyv.x, oyv.x, fyv.x, by.x);
                    vy.y = face_val_br<LIM>(cyv.y, oyv.y, fyv.y, by.y);
                    if (!top) {
                        vz.x = face_val_br<LIM>(czv.x, ozv.x, fzv.x, bz.x);
                        vz.y = face_val_br<LIM>(czv.y, ozv.y, fzv.y, bz.y);
                    } else {
                        vz.x = vz.y = T(0);
                    }
                }
                xp[q].x = mup * vx.x; xp[q].y = mup * vx.y;
                yp[q].x = mvp * vy.x; yp[q].y = mvp * vy.y;
                zp[q].x = top ? T(0) : mwp * vz.x;
                zp[q].y = top ? T(0) : mwp * vz.y;
                if (valid) {
                    const long long fs = (long long)nz * plane, ds = (long long)NT * fs;
                    // the record of field 2q+1 (and 2q+2) of this cell, in [NT][nz][ny][nx]
                    // (branches) and [3][NT][nz][ny][nx] (face values)
                    long long bi = (long long)(2 * q) * fs + (long long)k * plane + own;
                    ASUCA_BC(bi, (2 * q + 2 <= NT ? NT - 1 : NT) * fs, p.status);
                    uint8_t *br = p.branch + bi;
                    br[0] = (uint8_t)(bx.x | (by.x << 2) | (bz.x << 4));
                    if (2 * q + 2 <= NT) br[fs] = (uint8_t)(bx.y | (by.y << 2) | (bz.y << 4));
                    if (p.facev) {
                        T *fv = p.facev + bi;
                        fv[0] = vx.x;
                        fv[ds] = vy.x;
                        fv[2 * ds] = vz.x;
                        if (2 * q + 2 <= NT) {
                            fv[fs] = vx.y;
                            fv[ds + fs] = vy.y;
                            fv[2 * ds + fs] = vz.y;
                        }
                    }
                }
            } else {
                xp[q] = flux2(q, cxv, oxv, fxv, mup);
                yp[q] = flux2(q, cyv, oyv, fyv, mvp);
                if (!top) zp[q] = flux2(q, czv, ozv, fzv, mwp);
                else zp[q].x = zp[q].y = T(0);
            }
            ysm[(q * (TY + 1) + ty + 1) * TX + tx] = yp[q];
        }
        {
            // Edge faces as warp tasks: one per pair for the j0-1/2 faces of the
            // 32 columns, and the NPF x TY faces at i0-1/2 packed 32 to a task
            // (lane l takes row l % TY, as 32 is a multiple of TY).
            constexpr int NYT = NPF, NXT = (NPF * TY + 31) / 32;
            const bool ub = meb >= T(0), ul = mel >= T(0);
            const int bc = (ub ? 1 : 2) * YS + cx * XS, bo = (ub ? 2 : 1) * YS + cx * XS,
                      bf = (ub ? 0 : 3) * YS + cx * XS;
            const int lr = (er + 2) * YS;
            const int lc = lr + (ul ? 3 : 4) * XS, lo = lr + (ul ? 4 : 3) * XS, lf = lr + (ul ? 2 : 5) * XS;
#pragma unroll 1
            for (int w = warp; w < NYT + NXT; w += TY) {
                if (w < NYT) {
                    // flux at j0-1/2 for column lane: slot rows 0..3 (j0-2 .. j0+1)
                    ysm[(w * (TY + 1)) * TX + tx] = flux2(w, ld2(Sk, w, bc), ld2(Sk, w, bo), ld2(Sk, w, bf), meb);
                } else {
                    // flux at i0-1/2 for row er of pair q: slot columns 2..5 (i0-2 .. i0+1)
                    const int q = ((w - NYT) * 32 + lane) / TY;
                    if (q < NPF) xbs[q * TY + er] = flux2(q, ld2(Sk, q, lc), ld2(Sk, q, lo), ld2(Sk, q, lf), mel);
                }
            }
        }
        __syncthreads();

        // ---- divergence and RK combine: out = Y^n + ax dX + ay dY + az dZ (+ cdt tendency),
        // each step one FMA on an exact difference
        const T az = -cdt * p.rdz[k];
        // z flux difference F(k+1/2) - F(k-1/2): ahead minus carried upward,
        // carried minus ahead downward (the same operands either way)
        const T dzf0 = DOWN ? zlo0 - mwp : mwp - zlo0;
        const T out0 = fma(az, dzf0, fma(ay, mvp - mvm, fma(ax, mup - mum, yb0)));
        zlo0 = mwp;
        T2 out2[NPF];
#pragma unroll
        for (int q = 0; q < NPF; q++) {
            T2 xm;
            xm.x = __shfl_up_sync(0xffffffffu, xp[q].x, 1);
            xm.y = __shfl_up_sync(0xffffffffu, xp[q].y, 1);
            if (lane == 0) xm = xbs[q * TY + ty];
            const T2 ym = ysm[(q * (TY + 1) + ty) * TX + tx];
            if constexpr (PACK) {
                const float2 neg1 = make_float2(-1.f, -1.f);
                float2 o = __ffma2_rn(make_float2(ax, ax), __ffma2_rn(xm, neg1, xp[q]), yb[q]);
                o = __ffma2_rn(make_float2(ay, ay), __ffma2_rn(ym, neg1, yp[q]), o);
                o = __ffma2_rn(make_float2(az, az), DOWN ? __ffma2_rn(zp[q], neg1, zlo[q]) : __ffma2_rn(zlo[q], neg1, zp[q]),
                               o);
                out2[q] = o;
            } else {
                out2[q].x = fma(az, DOWN ? zlo[q].x - zp[q].x : zp[q].x - zlo[q].x,
                                fma(ay, yp[q].x - ym.x, fma(ax, xp[q].x - xm.x, yb[q].x)));
                out2[q].y = fma(az, DOWN ? zlo[q].y - zp[q].y : zp[q].y - zlo[q].y,
                                fma(ay, yp[q].y - ym.y, fma(ax, xp[q].y - xm.y, yb[q].y)));
            }
            zlo[q] = zp[q];
        }
        if (has_tend) {
            const long long fs = (long long)nz * plane;
            unsigned tb = (unsigned)k * plane + own;   // [F-1][nz][ny][nx]: fields at tb + f fs
            ASUCA_BC(tb, fs, p.status);
            const T *tk = p.tend + tb;
#pragma unroll
            for (int q = 0; q < NPF; q++) {
                out2[q].x = fma(cdt, tk[(long long)(2 * q) * fs], out2[q].x);
                if (2 * q + 2 <= NT) out2[q].y = fma(cdt, tk[(long long)(2 * q + 1) * fs], out2[q].y);
            }
        }
        if (Hook::active) {
            // the density result of the next march step, evaluated as that step
            // will (with the hook's coefficient for an own_rho hook, which also
            // receives this level's density so evaluated)
            const T hc = Hook::own_rho ? p.hcdt : cdt;
            const T hx = Hook::own_rho ? -hc * p.rdx : ax, hy = Hook::own_rho ? -hc * p.rdy : ay;
            const T rho_h = Hook::own_rho ? fma(-hc * p.rdz[k], dzf0, fma(hy, mvp - mvm, fma(hx, mup - mum, yb0))) : out0;
            T rho_next = T(0);
            if (t + 1 < nz) {
                const T az_n = -hc * p.rdz[level_of(t + 1)];
                rho_next = fma(az_n, DOWN ? mwp - nmwp : nmwp - mwp,
                               fma(hy, nmvp - nmvm, fma(hx, nmup - nmum, nrho)));
            }
            T out[NF];
            out[0] = out0;
#pragma unroll
            for (int q = 0; q < NPF; q++) {
                out[2 * q + 1] = out2[q].x;
                if (2 * q + 2 <= NT) out[2 * q + 2] = out2[q].y;
            }
            hook.template level<T, NF>(k, out, valid, rho_next, rho_h);
        }
        if (Hook::active && !Hook::keep_output) {
            // the hook took the level
        } else if (valid) {
            if (p.out_padded) {
                // the next stage reads phi = (rho phi) / rho, in pairs; the
                // density goes with the last pair (or a pair of its own)
                const T r = recip(out0);
                constexpr int NW = (NT & 1) ? NPF : NPF + 1;   // pairs written
                // the cell's first element; the pairs at + q q2 (+1 for the second value),
                // the periodic ghost copies at + gx, + gy (buffer: nz plev elements)
                long long oo = (long long)k * p.plev + (long long)(j + 2) * p.prow + 2 * (i + 4);
                ASUCA_BC(oo, (long long)nz * p.plev - (NW - 1) * q2 - 1, p.status);
                T *ob = p.yout[1] + oo;
                T2 v[NPF + 1];
#pragma unroll
                for (int q = 0; q < NPF; q++) {
                    if constexpr (PACK) {
                        v[q] = __fmul2_rn(out2[q], make_float2(r, r));
                    } else {
                        v[q].x = out2[q].x * r;
                        v[q].y = out2[q].y * r;
                    }
                }
                if (NT & 1) v[NPF - 1].y = out0;
                else {
                    v[NPF].x = out0;
                    v[NPF].y = T(0);
                }
#pragma unroll
                for (int q = 0; q < NW; q++) *reinterpret_cast<T2 *>(ob + q * q2) = v[q];
                if (ghost_x || ghost_y) {
                    long long gx = (i < 2) ? 2LL * nx : ((i >= nx - 2) ? -2LL * nx : 0);
                    long long gy = (j < 2) ? (long long)ny * p.prow : ((j >= ny - 2) ? -(long long)ny * p.prow : 0);
#ifdef ASUCA_BOUNDS_CHECK
                    {   // the ghost copies' first elements inside the buffer
                        long long ox = oo + gx, oy = oo + gy;
                        ASUCA_BC(ox, (long long)nz * p.plev - (NW - 1) * q2 - 1, p.status);
                        ASUCA_BC(oy, (long long)nz * p.plev - (NW - 1) * q2 - 1, p.status);
                        gx = ox - oo;
                        gy = oy - oo;
                    }
#endif
#pragma unroll
                    for (int q = 0; q < NW; q++) {
                        if (gx) *reinterpret_cast<T2 *>(ob + q * q2 + gx) = v[q];
                        if (gy) *reinterpret_cast<T2 *>(ob + q * q2 + gy) = v[q];
                    }
                }
            } else {
                unsigned o = (unsigned)k * plane + own;
                ASUCA_BC(o, (long long)nz * plane, p.status);
                p.yout[0][o] = out0;
#pragma unroll
                for (int q = 0; q < NPF; q++) {
                    p.yout[2 * q + 1][o] = out2[q].x;
                    if (2 * q + 2 <= NT) p.yout[2 * q + 2][o] = out2[q].y;
                }
            }
        }
        if (t + 1 < nz) advance();
    }
    if (Hook::active && !timed_out) hook.done(valid);

    if (timed_out) {
        if (tid == 0 && p.status) atomicCAS(p.status, 0, (int)ASUCA_ERR_TIMEOUT);
        // let the copies still in flight land (each wait bounded) before the
        // shared memory is released
        if (tma)
            for (int lev = seen; lev < issued; lev++)
                if (!mbar_wait(&bars[lev % D], (lev / D) & 1)) break;
    }
    if (!tma) cp_async_wait<0>();
    __syncthreads();
    return timed_out;
}

// A tile of a stage, its input layout chosen by the input (padded stage
// buffer: pairs; the caller's fields: raw).
template <typename T, int NF, int LIM, bool REC, int TYV = 8>
__device__ __forceinline__ bool stage_tile(const StageParams<T> &p, const CUtensorMap *tmap, int i0, int j0,
                                           unsigned char *smem_raw, const CUtensorMap *umaps = nullptr) {
    NoHook h;
    if (p.tma_in) return stage_tile_h<T, NF, LIM, REC, TYV, false, NoHook, LAYOUT_PAIR>(p, tmap, i0, j0, smem_raw, h);
    return stage_tile_h<T, NF, LIM, REC, TYV, false, NoHook, LAYOUT_RAW>(p, tmap, i0, j0, smem_raw, h, umaps);
}

template <typename T, int NF, int LIM, bool REC, int TYV, int LAY>
__global__ void __launch_bounds__(32 * TYV, StageShape<T, NF, TYV>::MIN_BLOCKS)
    stage_kernel(const __grid_constant__ StageParams<T> p) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    NoHook h;
    (void)stage_tile_h<T, NF, LIM, REC, TYV, false, NoHook, LAY>(p, &p.tmap, blockIdx.x * StageShape<T, NF, TYV>::TX,
                                                                blockIdx.y * TYV, smem_raw, h);
}

template <typename T, int NF, int LIM, bool REC, int TYV, int LAY>
static cudaError_t launch_lay(const StageParams<T> &p, cudaStream_t s) {
    using S = StageShape<T, NF, TYV>;
    static std::atomic<unsigned long long> attr_done{0};   // devices whose attribute is set
    const cudaError_t e = set_smem_once(stage_kernel<T, NF, LIM, REC, TYV, LAY>, (int)S::SMEM_BYTES, attr_done);
    if (e != cudaSuccess) return e;
    dim3 block(S::TX, S::TY);
    dim3 grid((p.nx + S::TX - 1) / S::TX, (p.ny + S::TY - 1) / S::TY);
    stage_kernel<T, NF, LIM, REC, TYV, LAY><<<grid, block, S::SMEM_BYTES, s>>>(p);
    return cudaGetLastError();
}

template <typename T, int NF, int LIM, bool REC, int TYV>
static cudaError_t launch_rec(const StageParams<T> &p, cudaStream_t s) {
    if (p.tma_in) return launch_lay<T, NF, LIM, REC, TYV, LAYOUT_PAIR>(p, s);
    return launch_lay<T, NF, LIM, REC, TYV, LAYOUT_RAW>(p, s);
}

// branch recording (the adjoint's forward pass) is instantiated for 4- and
// 8-row tiles
template <typename T, int NF, int LIM, int TYV>
static cudaError_t launch_lim(const StageParams<T> &p, cudaStream_t s) {
    if (p.branch) {
        if constexpr (TYV == 4 || TYV == 8) return launch_rec<T, NF, LIM, true, TYV>(p, s);
        else return cudaErrorInvalidValue;
    }
    return launch_rec<T, NF, LIM, false, TYV>(p, s);
}

template <typename T, int NF, int TYV>
static cudaError_t launch_nf(const StageParams<T> &p, cudaStream_t s) {
    switch (p.lim) {
        case ASUCA_LIM_KOREN: return launch_lim<T, NF, ASUCA_LIM_KOREN, TYV>(p, s);
        case ASUCA_LIM_LINEAR: return launch_lim<T, NF, ASUCA_LIM_LINEAR, TYV>(p, s);
        case ASUCA_LIM_UPWIND1: return launch_lim<T, NF, ASUCA_LIM_UPWIND1, TYV>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int TYV>
cudaError_t launch_stage_ty(const StageParams<T> &p, int nf, cudaStream_t s) {
    switch (nf) {
        case 2: return launch_nf<T, 2, TYV>(p, s);
        case 3: return launch_nf<T, 3, TYV>(p, s);
        case 4: return launch_nf<T, 4, TYV>(p, s);
        case 5: return launch_nf<T, 5, TYV>(p, s);
        case 6: return launch_nf<T, 6, TYV>(p, s);
        case 7: return launch_nf<T, 7, TYV>(p, s);
        case 8: return launch_nf<T, 8, TYV>(p, s);
        case 9: return launch_nf<T, 9, TYV>(p, s);
        case 10: return launch_nf<T, 10, TYV>(p, s);
        default: return cudaErrorInvalidValue;
    }
}

static inline PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
    }
    return fn;
}

template <typename T>
cudaError_t encode_stage_map(CUtensorMap *map, void *base, int nf, int nx, int ny, int nz, int ty) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    if (nf < 2) return cudaErrorInvalidValue;
    using S = StageShape<T, 2>;   // SX does not depend on the field count or the tile height
    const long long P = padded_pitch(nx);
    // the pair layout as a 4D tensor (2 pitch elements, pairs, rows, levels);
    // the map covers the phi pairs (the density, in the last pair or a pair of
    // its own, stays in the buffer for the adjoint)
    const int np = pair_count(nf), npf = (nf - 1 + 1) / 2;
    const cuuint64_t dims[4] = {(cuuint64_t)(2 * P), (cuuint64_t)npf, (cuuint64_t)(ny + 4), (cuuint64_t)nz};
    const cuuint64_t strides[3] = {(cuuint64_t)(2 * P * sizeof(T)), (cuuint64_t)(2 * P * np * sizeof(T)),
                                   (cuuint64_t)(2 * P * np * (ny + 4) * sizeof(T))};
    const cuuint32_t box[4] = {(cuuint32_t)(2 * S::SX), (cuuint32_t)npf, (cuuint32_t)(ty + 4), 1u};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    CUresult r = enc(map, sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 4,
                     base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <typename T>
cudaError_t encode_user_maps(CUtensorMap *maps, const void *rho, const void *rhotheta, const void *rhoq, int ntr,
                             int nx, int ny, int nz, int ty) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return cudaErrorNotSupported;
    using S = StageShape<T, 2>;
    const CUtensorMapDataType dt = sizeof(T) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)(ntr > 0 ? ntr : 1)};
    const cuuint64_t strides[3] = {(cuuint64_t)nx * sizeof(T), (cuuint64_t)nx * ny * sizeof(T),
                                   (cuuint64_t)nx * ny * (cuuint64_t)nz * sizeof(T)};
    const cuuint32_t box[4] = {(cuuint32_t)S::SX, (cuuint32_t)(ty + 4), 1u, (cuuint32_t)(ntr > 0 ? ntr : 1)};
    const cuuint32_t estr[4] = {1u, 1u, 1u, 1u};
    const void *base[3] = {rho, rhotheta, rhoq};
    for (int q = 0; q < 3; q++) {
        if (q == 2 && ntr == 0) {
            std::memset(&maps[q], 0, sizeof(CUtensorMap));
            continue;
        }
        const cuuint32_t rank = q == 2 ? 4u : 3u;
        CUresult r = enc(&maps[q], dt, rank, const_cast<void *>(base[q]), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
}


}  // namespace asuca
