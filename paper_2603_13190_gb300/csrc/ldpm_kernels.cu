// ldpm_kernels.cu -- sm_103a kernels of the LDPM explicit central-difference step.
//
// One step (paper Sec. 3, central difference with lumped mass) is two launches.  Between steps the
// state is kept drifted: q_{n+1} and v_{n+1/2} (and f_n); kick_kernel / unkick_kernel convert from /
// to the whole-step state q_n, v_n at the API boundary.
//   facet_kernel / facet_warp_kernel
//                  per facet: rigid-body jump and strain (Sec. 2, Eq. (1)), per-tetrahedron
//                  volumetric strain (App. A.2 e_V), the Appendix A law, force A P t; then per
//                  tetrahedron vertex the fixed-order sum of its 6 facets' forces and moments
//                  (the tetrahedron's share of Eq. (2a)-(2b)).  The warp variant (one 8-tetrahedron
//                  tile per warp) runs the FP32 pass, the block variant the FP64 pass and larger tiles;
//   gather_kernel  per particle: fixed-order sum of its (tetrahedron, vertex) shares, then the second
//                  half kick of this step, the energy increments, and the first half kick and drift
//                  of the next step.
// No tensor cores (no dense contraction), no float atomics.  The passes are bound by memory latency
// and instruction issue (the FP64 ones by the FP64 pipe) well before HBM bandwidth.
#include <algorithm>
#include <cstdint>
#include <type_traits>

#include <cuda_runtime.h>

#include "ldpm_device.cuh"
#include "ldpm_internal.h"

namespace ldpm {
namespace {

// ------------------------------------------------------------------------------------------------
// Facet pass.  A block owns TETS consecutive tetrahedra (12 * TETS facets, one thread each).
//   phase A  4 threads per tetrahedron gather the vertex records (mixed mode: the 96-byte FP32
//            mirror, two-float differences; FP64 mode: the 128-byte FP64 record) and write the
//            differences to vertex 0 of the tetrahedron to shared memory, then the tetrahedron's
//            volumetric strain;
//   phase B  one thread per facet: kinematics, law, force, and its contributions to its two
//            vertices (force and moment about each);
//   phase C  12 threads per tetrahedron: thread s sums components 2(s%3), 2(s%3)+1 of vertex s/3
//            over the vertex's 6 facets in a fixed order (its 3 edges ascending, each edge's two
//            facets in slot order).
// Shared-memory rows are 16-byte aligned and accessed with 128/64-bit vectors (the pass is bound by
// L1/shared-memory wavefronts before HBM).  The facet's geometry and history are loaded into
// registers before phase A so their HBM latency overlaps the gathers.
// ------------------------------------------------------------------------------------------------
constexpr int kRow = 16;  // vertex row: dx(3) du(3) dv(3) theta(3) omega(3) pad
constexpr int kCon = 12;  // facet row: contribution to vertex a (6), to vertex b (6)
// Row strides in elements: with 16-byte accesses, 8 consecutive rows must start in distinct 4-bank
// groups (stride = 4 mod 8 banks for floats is 20 or 12 words; doubles use 36 and 28 words).
template <class R>
struct Stride {
    static constexpr int row = sizeof(R) == 4 ? 20 : 18;
    static constexpr int con = sizeof(R) == 4 ? 12 : 14;
};

// Loads of data that the persistent step kernel writes during its own launch (particle records,
// history, vertex shares, the step counter).  With PERSIST they are explicit weak global loads
// (ld.global.ca): never the read-only non-coherent path a compiler may pick for const __restrict__
// pointers, which is valid only for data that no thread writes during the launch.  Values written
// by other blocks become visible through the grid barrier's fences.
template <bool PERSIST, class T>
__device__ __forceinline__ T ld_live(const T *p)
{
    if constexpr (PERSIST)
        return __ldca(p);
    else
        return *p;
}
template <bool PERSIST>
__device__ __forceinline__ double4a ld_live(const double4a *p)
{
    if constexpr (PERSIST) {
        const double2 a = __ldca(reinterpret_cast<const double2 *>(p));
        const double2 b = __ldca(reinterpret_cast<const double2 *>(p) + 1);
        return double4a{a.x, a.y, b.x, b.y};
    } else {
        return *p;
    }
}

// Staging of one tetrahedron vertex (lane4 = 4 * tetrahedron + vertex within the tile; all 32 lanes
// of the warp take part, the shuffles stay within each tetrahedron's 4 lanes): the particle record,
// differences to the tetrahedron's vertex 0 into shared row sv[lane4], and e_V of the tetrahedron.
template <class R, int MODE, bool PERSIST = false>
__device__ __forceinline__ void stage_vertex(const DeviceModel &m, const void *__restrict__ vsrc, int64_t tet0,
                                             int lane4, R (*sv)[Stride<R>::row], R *seV, int *sok)
{
    constexpr int E = 16 / (int)sizeof(R);
    const LawConst<R> *__restrict__ lawc = static_cast<const LawConst<R> *>(m.law);
    (void)lawc;
    const int jt = lane4 >> 2, vi = lane4 & 3;
    const int64_t tt = tet0 + jt;
    int p = -1;
    if (tt < m.T) p = reinterpret_cast<const int *>(m.tet)[4 * tt + vi];
    const int base = (threadIdx.x & 31) & ~3;
    R o[kRow];
    if constexpr (sizeof(R) == 4) {
        // mirror: x_hi 0..2, x_lo 3..5, u_hi 6..8, u_lo 9..11, theta 12..14, v 15..17, omega 18..20.
        // (a_hi - b_hi) + (a_lo - b_lo) carries FP32 relative accuracy of the difference itself.
        const float *src = static_cast<const float *>(vsrc);
        float rec[24];
        if (p >= 0) {
            const float4 *r4 = reinterpret_cast<const float4 *>(src + kMirror * (int64_t)p);
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                const float4 w = ld_live<PERSIST>(r4 + k);
                rec[4 * k] = w.x;
                rec[4 * k + 1] = w.y;
                rec[4 * k + 2] = w.z;
                rec[4 * k + 3] = w.w;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 24; ++k) rec[k] = 0.0f;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float x0h = __shfl_sync(0xffffffffu, rec[k], base);
            const float x0l = __shfl_sync(0xffffffffu, rec[3 + k], base);
            const float u0h = __shfl_sync(0xffffffffu, rec[6 + k], base);
            const float u0l = __shfl_sync(0xffffffffu, rec[9 + k], base);
            const float v0 = __shfl_sync(0xffffffffu, rec[15 + k], base);
            o[k] = (rec[k] - x0h) + (rec[3 + k] - x0l);
            o[3 + k] = (rec[6 + k] - u0h) + (rec[9 + k] - u0l);
            o[6 + k] = rec[15 + k] - v0;
            o[9 + k] = rec[12 + k];
            o[12 + k] = rec[18 + k];
        }
    } else {
        // FP64 record: x 0..2, u 3..5, theta 6..8, v 9..11, omega 12..14
        const double *src = static_cast<const double *>(vsrc);
        double rec[16];
        if (p >= 0) {
            const double2 *r2 = reinterpret_cast<const double2 *>(src + 16 * (int64_t)p);
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const double2 w = ld_live<PERSIST>(r2 + k);
                rec[2 * k] = w.x;
                rec[2 * k + 1] = w.y;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) rec[k] = 0.0;
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const double x0 = __shfl_sync(0xffffffffu, rec[k], base);
            const double u0 = __shfl_sync(0xffffffffu, rec[3 + k], base);
            const double v0 = __shfl_sync(0xffffffffu, rec[9 + k], base);
            o[k] = rec[k] - x0;
            o[3 + k] = rec[3 + k] - u0;
            o[6 + k] = rec[9 + k] - v0;
            o[9 + k] = rec[6 + k];
            o[12 + k] = rec[12 + k];
        }
    }
    if (MODE == FACET_METRIC) {  // whole-step state: u_n = u_{n+1} - dt v_{n+1/2}, same for theta
        const R dtm = lawc[m.tile_spec ? m.tile_spec[tet0 / 32] : 0].dt;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            o[3 + k] -= dtm * o[6 + k];
            o[9 + k] -= dtm * o[12 + k];
        }
    }
    o[15] = R(0);
#pragma unroll
    for (int k = 0; k < kRow; k += E) VecT<R>::put(&sv[lane4][k], &o[k]);
    // e_V = (1/3) div u of the linear tetrahedron.  With D = [dx1 dx2 dx3], grad N_i (i = 1..3)
    // are the rows of D^-1 = [dx2 x dx3; dx3 x dx1; dx1 x dx2] / det D, and vertex 0 carries no
    // displacement difference.  Lane i >= 1 forms its own term du_i . (dx_i1 x dx_i2).
    const V3<R> dxs = {o[0], o[1], o[2]};
    const V3<R> dus = {o[3], o[4], o[5]};
    const int i1 = vi == 3 ? 1 : vi + 1;
    const int i2 = i1 == 3 ? 1 : i1 + 1;
    V3<R> a1, a2;
    a1.x = __shfl_sync(0xffffffffu, dxs.x, base + i1);
    a1.y = __shfl_sync(0xffffffffu, dxs.y, base + i1);
    a1.z = __shfl_sync(0xffffffffu, dxs.z, base + i1);
    a2.x = __shfl_sync(0xffffffffu, dxs.x, base + i2);
    a2.y = __shfl_sync(0xffffffffu, dxs.y, base + i2);
    a2.z = __shfl_sync(0xffffffffu, dxs.z, base + i2);
    const V3<R> cr = cross(a1, a2);
    R term = vi == 0 ? R(0) : dot(dus, cr);
    R det = vi == 0 ? R(0) : dot(dxs, cr);
    term += __shfl_xor_sync(0xffffffffu, term, 1);
    term += __shfl_xor_sync(0xffffffffu, term, 2);
    det = __shfl_sync(0xffffffffu, det, base + 1);
    if (vi == 0) {
        seV[jt] = (p >= 0 && det != R(0)) ? term / (R(3) * det) : R(0);
        sok[jt] = p >= 0;
    }
}

// One facet (tetrahedron j of the tile, slot 0..11, global facet f): kinematics, law, history, force,
// and its contributions to its two vertices in cs[12] (zeros when the facet is not live).
// S1: one specimen in mixed mode, law constants taken from m.law1 (the kernel parameters) instead of
// the global array; see facet_warp_kernel.
template <class R, int MODE, bool PF, bool S1 = false>
__device__ __forceinline__ void facet_one(const DeviceModel &m, int64_t tet0, int j, int slot, int64_t f, bool live,
                                          const R4<R> &g, const R4<R> &h, const R4<R> &pp,
                                          const R (*sv)[Stride<R>::row], const R *seV, R cs[12],
                                          const LawConst<R> *lbatch = nullptr)
{
    using T4 = R4<R>;
    constexpr int E = 16 / (int)sizeof(R);
    T4 *__restrict__ hout = static_cast<T4 *>(m.hist_out ? m.hist_out : m.hist);  // the new history
    T4 *__restrict__ fout = static_cast<T4 *>(m.fout);
    const LawConst<R> *__restrict__ lawc = static_cast<const LawConst<R> *>(m.law);
    (void)pp;
    if (!live) {
#pragma unroll
    for (int k = 0; k < 12; ++k) cs[k] = R(0);
    } else {
    const int e = slot >> 1;
    const int va = (0x211000 >> (4 * e)) & 0xF;
    const int vb = (0x332321 >> (4 * e)) & 0xF;
    R A[kRow], B[kRow];
#pragma unroll
    for (int k = 0; k < kRow; k += E) {
        VecT<R>::get(&A[k], &sv[4 * j + va][k]);
        VecT<R>::get(&B[k], &sv[4 * j + vb][k]);
    }
    const V3<R> d = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
    const R inv_l = rsqrt_(dot(d, d));
    const R l = dot(d, d) * inv_l;
    const V3<R> n = inv_l * d;
    V3<R> mt, lt;
    tangent_frame(n, mt, lt);
    const V3<R> ca = {g.x, g.y, g.z};
    const V3<R> cb = ca - d;
    R tN, tM, tL, emax;
    const LawConst<R> *lsrc;
    if (lbatch) {  // the batch kernel's parameters
        lsrc = lbatch;
    } else if constexpr (S1 && sizeof(R) == 4) {
        lsrc = reinterpret_cast<const LawConst<R> *>(&m.law1);
    } else {
        const int sp = m.tile_spec ? m.tile_spec[tet0 / 32] : 0;  // specimens are padded to 32 tetrahedra
        lsrc = lawc + sp;
    }
    LawConst<R> cpf;
    if constexpr (PF) cpf = facet_params(*lsrc, pp.x, pp.y, pp.z);
    const LawConst<R> &c = PF ? cpf : *lsrc;
    if (MODE == FACET_FROM_HIST) {
        tN = h.x;
        tM = h.y;
        tL = h.z;
    } else {
        const V3<R> thA = {A[9], A[10], A[11]}, thB = {B[9], B[10], B[11]};
        const V3<R> du = {B[3] - A[3], B[4] - A[4], B[5] - A[5]};
        const V3<R> jump = du + cross(thB, cb) - cross(thA, ca);
        const V3<R> e3 = {dot(n, jump) * inv_l, dot(mt, jump) * inv_l, dot(lt, jump) * inv_l};
        if (MODE == FACET_ELASTIC) {
            tN = c.E0 * e3.x;
            tM = c.alpha * c.E0 * e3.y;
            tL = c.alpha * c.E0 * e3.z;
        } else if (MODE == FACET_METRIC) {
            // crack opening from the inelastic part of the jump: w_N = l <e_N - t_N / E0>,
            // w_T = l (e_T - t_T / (alpha E0)) (u here is already u_n)
            R wn = e3.x - h.x / c.E0;
            wn = wn > R(0) ? wn : R(0);
            const R aE = c.alpha * c.E0;
            const R wm = e3.y - h.y / aE, wl = e3.z - h.z / aE;
            T4 o4;
            o4.x = l * sqrt(wn * wn + wm * wm + wl * wl);
            o4.y = seV[j];
            o4.z = R(0);
            o4.w = R(0);
            fout[f] = o4;
            tN = tM = tL = R(0);
        } else {
            const V3<R> omA = {A[12], A[13], A[14]}, omB = {B[12], B[13], B[14]};
            const V3<R> dv = {B[6] - A[6], B[7] - A[7], B[8] - A[8]};
            const V3<R> djump = dv + cross(omB, cb) - cross(omA, ca);
            const R sdt = c.dt * inv_l;
            const V3<R> de3 = {dot(n, djump) * sdt, dot(mt, djump) * sdt, dot(lt, djump) * sdt};
            tN = h.x;
            tM = h.y;
            tL = h.z;
            emax = h.w;
            facet_law(c, l, e3, de3, seV[j], tN, tM, tL, emax);
            T4 hn;
            hn.x = tN;
            hn.y = tM;
            hn.z = tL;
            hn.w = emax;
            hout[f] = hn;
        }
    }
    const R Ar = g.w;
    const V3<R> F = {Ar * (tN * n.x + tM * mt.x + tL * lt.x), Ar * (tN * n.y + tM * mt.y + tL * lt.y),
                     Ar * (tN * n.z + tM * mt.z + tL * lt.z)};
    if (MODE == FACET_FROM_HIST) {  // per-facet force, kept only for ldpm_facet_forces
        T4 Fo;
        Fo.x = F.x;
        Fo.y = F.y;
        Fo.z = F.z;
        Fo.w = R(0);
        fout[f] = Fo;
    }
    // vertex a receives +F and the moment c_a x F about itself; vertex b -F and c_b x (-F)
    const V3<R> Ma = cross(ca, F);
    const V3<R> Mb = cross(cb, F);
    cs[0] = F.x;
    cs[1] = F.y;
    cs[2] = F.z;
    cs[3] = Ma.x;
    cs[4] = Ma.y;
    cs[5] = Ma.z;
    cs[6] = -F.x;
    cs[7] = -F.y;
    cs[8] = -F.z;
    cs[9] = -Mb.x;
    cs[10] = -Mb.y;
    cs[11] = -Mb.z;
    }
}

// Per tetrahedron vertex v = slot / 3, components 2 q, 2 q + 1 (q = slot % 3): the fixed-order sum over
// its 3 edges (ascending), each edge's two facets in slot order.
template <class R>
__device__ __forceinline__ void vertex_sum(const DeviceModel &m, int64_t tet0, int j, int slot,
                                           const R (*scon)[Stride<R>::con])
{
    using V2 = typename VecT<R>::v2;
    R *__restrict__ tvc = static_cast<R *>(m.tvc);
    const int v = slot / 3;
    const int q = slot - 3 * v;
    const int edges = (int)((0x542531430210ull >> (12 * v)) & 0xFFF);
    const int sides = (0xEC8 >> (3 * v)) & 0x7;  // v0: 000, v1: 001, v2: 011, v3: 111
    R s0 = R(0), s1 = R(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int e2 = (edges >> (4 * k)) & 0xF;
        const int col = (((sides >> k) & 1) ? 6 : 0) + 2 * q;
        const V2 w0 = *reinterpret_cast<const V2 *>(&scon[12 * j + 2 * e2][col]);
        const V2 w1 = *reinterpret_cast<const V2 *>(&scon[12 * j + 2 * e2 + 1][col]);
        s0 += w0.x;
        s1 += w0.y;
        s0 += w1.x;
        s1 += w1.y;
    }
    *reinterpret_cast<V2 *>(tvc + (tet0 + j) * 24 + 6 * v + 2 * q) = V2{s0, s1};
}

// One tile of TETS tetrahedra run by a block of 12 TETS threads (one facet each): phases A-C above.
// PF: the facet's own E0, alpha, sigma_t (m.pf) replace the material's in the law.  PERSIST: called
// from the persistent step kernel (live data through ld_live; the block's shared rows are reused for
// the next tile after the closing barrier).
template <class R, int MODE, int TETS, bool PF, bool PERSIST>
__device__ __forceinline__ void facet_block_tile(const DeviceModel &m, const void *__restrict__ vsrc, int64_t tet0,
                                                 R (*sv)[Stride<R>::row], R (*scon)[Stride<R>::con], R *seV,
                                                 int *sok)
{
    using T4 = R4<R>;
    constexpr int E = 16 / (int)sizeof(R);  // elements per 16-byte shared-memory vector
    const T4 *__restrict__ geo = static_cast<const T4 *>(m.geo);
    const T4 *__restrict__ hist = static_cast<const T4 *>(m.hist);
    const int tid = threadIdx.x;

    // ---- prefetch this thread's facet data
    const int j = tid / 12;
    const int slot = tid - 12 * j;
    const int64_t f = tet0 * 12 + tid;
    const bool valid = tet0 + j < m.T;
    T4 g{}, h{}, pp{};
    if (valid) {
        g = geo[f];
        if (MODE != FACET_ELASTIC) h = ld_live<PERSIST>(hist + f);
        if (PF) pp = static_cast<const T4 *>(m.pf)[f];
    }

    // ---- phase A: vertex records -> shared memory, e_V per tetrahedron
    if (tid < 4 * TETS) stage_vertex<R, MODE, PERSIST>(m, vsrc, tet0, tid, sv, seV, sok);
    __syncthreads();

    // ---- phase B: one facet
    const bool live = valid && sok[j];
    R cs[12];
    facet_one<R, MODE, PF>(m, tet0, j, slot, f, live, g, h, pp, sv, seV, cs);
#pragma unroll
    for (int k = 0; k < kCon; k += E) VecT<R>::put(&scon[tid][k], &cs[k]);
    __syncthreads();

    // ---- phase C
    if (live && MODE != FACET_METRIC) vertex_sum<R>(m, tet0, j, slot, scon);
    if (PERSIST) __syncthreads();
}

template <class R, int MODE, int TETS, bool PF>
__global__ void __launch_bounds__(12 * TETS) facet_kernel(DeviceModel m, const void *__restrict__ vsrc)
{
    __shared__ alignas(16) R sv[TETS * 4][Stride<R>::row];
    __shared__ alignas(16) R scon[12 * TETS][Stride<R>::con];
    __shared__ R seV[TETS];
    __shared__ int sok[TETS];
    const int64_t tet0 = (int64_t)blockIdx.x * TETS;
    if (MODE == FACET_STEP && blockIdx.x == 0 && threadIdx.x == 0) *m.step += 1;
    facet_block_tile<R, MODE, TETS, PF, false>(m, vsrc, tet0, sv, scon, seV, sok);
}

// Warp-tile variant of facet_kernel: every warp owns a tile of 8 tetrahedra and runs phases A-C on it
// alone (lane = vertex in phase A, three facets per lane in phase B, three vertex sums per lane in
// phase C), synchronising only within the warp, so each warp's record gathers are in flight
// independently of the other warps.  Same arithmetic and summation order as facet_kernel<.., 8, ..>.
// The facets' contributions are stored vertex-major: plane s (0..5) holds, for every vertex of the
// tile, the contribution of the s-th facet in that vertex's fixed summation order (its 3 edges
// ascending, each edge's two facets in slot order), 6 values per vertex.  The vertex sum of
// components 2q, 2q+1 of vertex v of tetrahedron j (task t = 12 j + 3 v + q) then reads word 2t of
// each plane: contiguous for the lanes, free of bank conflicts.  Planes are kPlane words apart (192
// plus 2, so that the facets' stores into different planes fall on different banks).
// With one specimen (S1) the law constants are read from the kernel's own parameters (m is a
// __grid_constant__, so taking its address makes no copy): there they are operands of the
// instructions that use them, where the global array costs a load per use and facet (measured on
// GB300 in the loaded state of 1.82M facets: 43.1 us against 45.2 us).
constexpr int kTileTets = 8;
constexpr int kPlane = 6 * 4 * kTileTets + 2;
// One 8-tetrahedron tile of the facet pass, run by one warp on its own shared rows: phases A-C below.
// PERSIST: called from the persistent step kernel (live data through ld_live).
template <class R, int MODE, bool PF, bool S1, bool PERSIST>
__device__ __forceinline__ void facet_tile(const DeviceModel &m, const void *__restrict__ vsrc, int64_t tet0,
                                           int lane, R (*sv)[Stride<R>::row], R *spl, R *seV, int *sok,
                                           const LawConst<R> *lbatch = nullptr)
{
    using T4 = R4<R>;
    using V2 = typename VecT<R>::v2;
    const T4 *__restrict__ geo = static_cast<const T4 *>(m.geo);
    const T4 *hist = static_cast<const T4 *>(m.hist);
    // ---- prefetch the lane's three facets
    T4 g[3] = {}, h[3] = {}, pp[3] = {};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int fi = lane + 32 * i;
        const int64_t f = tet0 * 12 + fi;
        if (tet0 + fi / 12 < m.T) {
            g[i] = geo[f];
            if (MODE != FACET_ELASTIC) h[i] = ld_live<PERSIST>(hist + f);
            if (PF) pp[i] = static_cast<const T4 *>(m.pf)[f];
        }
    }
    // ---- phase A
    stage_vertex<R, MODE, PERSIST>(m, vsrc, tet0, lane, sv, seV, sok);
    __syncwarp();
    // ---- phase B
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const int fi = lane + 32 * i;
        const int j = fi / 12;
        const bool live = tet0 + j < m.T && sok[j];
        const int slot = fi - 12 * j;
        R cs[12];
        facet_one<R, MODE, PF, S1>(m, tet0, j, slot, tet0 * 12 + fi, live, g[i], h[i], pp[i], sv, seV, cs, lbatch);
        if (MODE != FACET_METRIC) {
            // edge e = slot / 2 joins local vertices va < vb; it is the ka-th edge of va and the kb-th
            // of vb (ascending), so this facet is entry 2 ka + slot % 2 of va's order, 2 kb + slot % 2 of vb's
            const int e = slot >> 1, sw = slot & 1;
            const int va = (0x211000 >> (4 * e)) & 0xF, vb = (0x332321 >> (4 * e)) & 0xF;
            const int ka = (0x221210 >> (4 * e)) & 0xF, kb = (0x211000 >> (4 * e)) & 0xF;
            R *da = spl + (2 * ka + sw) * kPlane + 6 * (4 * j + va);
            R *db = spl + (2 * kb + sw) * kPlane + 6 * (4 * j + vb);
#pragma unroll
            for (int c = 0; c < 6; c += 2) {
                *reinterpret_cast<V2 *>(da + c) = V2{cs[c], cs[c + 1]};
                *reinterpret_cast<V2 *>(db + c) = V2{cs[6 + c], cs[6 + c + 1]};
            }
        }
    }
    __syncwarp();
    // ---- phase C: task t = 12 j + 3 v + q sums components 2q, 2q+1 of vertex v over the 6 planes
    if (MODE != FACET_METRIC) {
        R *__restrict__ tvc = static_cast<R *>(m.tvc);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const int t = lane + 32 * i;
            const int j = t / 12;
            if (tet0 + j < m.T && sok[j]) {
                R s0 = R(0), s1 = R(0);
#pragma unroll
                for (int sp = 0; sp < 6; ++sp) {
                    const V2 x = *reinterpret_cast<const V2 *>(spl + sp * kPlane + 2 * t);
                    s0 += x.x;
                    s1 += x.y;
                }
                *reinterpret_cast<V2 *>(tvc + tet0 * 24 + 2 * t) = V2{s0, s1};
            }
        }
    }
    __syncwarp();  // the warp's shared rows may be reused for another tile
}

// Mixed mode: capped at 80 registers (12 blocks of 2 warps per SM); without the cap the multi-specimen
// instantiation took 93 registers and ran 8 % slower on the 97.7M-facet batch (GB300, side by side).
template <class R, int MODE, int WPB, bool PF, bool S1>
__global__ void __launch_bounds__(32 * WPB, sizeof(R) == 4 ? 12 : 1)
    facet_warp_kernel(const __grid_constant__ DeviceModel m, const void *__restrict__ vsrc)
{
    constexpr int TETS = kTileTets;
    __shared__ alignas(16) R sv_[WPB][TETS * 4][Stride<R>::row];
    __shared__ alignas(16) R spl_[WPB][6 * kPlane];
    __shared__ R seV_[WPB][TETS];
    __shared__ int sok_[WPB][TETS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tet0 = ((int64_t)blockIdx.x * WPB + w) * TETS;
    if (MODE == FACET_STEP && blockIdx.x == 0 && threadIdx.x == 0) *m.step += 1;
    if (tet0 >= m.T) return;  // whole warp (T is a multiple of the tile)
    facet_tile<R, MODE, PF, S1, false>(m, vsrc, tet0, lane, sv_[w], spl_[w], seV_[w], sok_[w]);
}

// The same for a batch of specimens, their law constants in the kernel parameters: a block of WPB
// 8-tetrahedron tiles (16 tetrahedra) lies within one specimen, found from the block index alone by
// a search over the specimens' first tetrahedra (all in the parameters), so the constants are read
// at a block-uniform index.
template <int MODE, int WPB, bool PF>
__global__ void __launch_bounds__(32 * WPB, 12)
    facet_warp_batch_kernel(const __grid_constant__ DeviceModel m, const void *__restrict__ vsrc,
                            const __grid_constant__ BatchLaw bl)
{
    static_assert(WPB * kTileTets <= 32 && 32 % (WPB * kTileTets) == 0, "a block within one 32-tetrahedron unit");
    constexpr int TETS = kTileTets;
    __shared__ alignas(16) float sv_[WPB][TETS * 4][Stride<float>::row];
    __shared__ alignas(16) float spl_[WPB][6 * kPlane];
    __shared__ float seV_[WPB][TETS];
    __shared__ int sok_[WPB][TETS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t tet0 = ((int64_t)blockIdx.x * WPB + w) * TETS;
    const int32_t tb = (int32_t)blockIdx.x * (WPB * TETS);
    int lo = 0, hi = bl.n;  // bl.t0[lo] <= tb < bl.t0[hi]
#pragma unroll
    for (int it = 0; it < 7; ++it) {  // 2^7 > kParamSpecimens
        const int mid = (lo + hi) >> 1;
        if (hi - lo > 1) {
            if (bl.t0[mid] <= tb)
                lo = mid;
            else
                hi = mid;
        }
    }
    if (MODE == FACET_STEP && blockIdx.x == 0 && threadIdx.x == 0) *m.step += 1;
    if (tet0 >= m.T) return;  // whole warp (T is a multiple of the tile)
    facet_tile<float, MODE, PF, false, false>(m, vsrc, tet0, lane, sv_[w], spl_[w], seV_[w], sok_[w], &bl.law[lo]);
}

// ------------------------------------------------------------------------------------------------
// Particle pass.  A group of LPP lanes owns one particle: it sums the particle's (tetrahedron,
// vertex) contributions in CSR order (Eq. (2a)-(2b)), reduces across the group by halving exchanges,
// after which six lanes of the group hold components 0..5 and update one DOF each.  With LPP = 8 a
// warp updates 4 particles per instruction.
// The particle's own records (mass, constraint, q, v, f_n) do not depend on the contributions and are
// loaded before the sum, so their latency overlaps the CSR gather.
// FP64 mode: everything is FP64.  Mixed mode: the shares are FP32 (each the sum of a tetrahedron's 6
// FP32 facet terms at one vertex); the particle sums of the shares are float-float (48 mantissa bits;
// components paired in packed FP32 instructions), converted to FP64 once; the velocity and
// displacement updates are FP64; the energy increments (trapezoid products with v_{n+1/2} and their
// 6-DOF sums) are float-float, scaled by dt/2 and added into the FP64 accumulators with one FP64 FMA
// each.  The GB300 FP64 pipe issues one warp instruction per ~64 cycles per sub-partition, so the
// compensated sums run on the FP32 pipe; FP32 <-> FP64 conversions are integer operations.
// ------------------------------------------------------------------------------------------------
// One group of LPP lanes, particle p (all 32 lanes of the warp take part in its shuffles).
template <class R, int MODE, int LPP, bool PERSIST>
__device__ __forceinline__ void gather_group(const DeviceModel &m, int64_t p, int lane, double *__restrict__ out6)
{
    static_assert(LPP == 8 || LPP == 16 || LPP == 32, "lanes per particle");
    constexpr bool kMixed = sizeof(R) == 4;
    const int32_t *__restrict__ ent = static_cast<const int32_t *>(m.ent);
    const R *tvc = static_cast<const R *>(m.tvc);
    const int sub = lane & (LPP - 1);
    const bool valid = p < m.N;
    // after the group's reduction, lanes 0..5 (mixed: pair_halving_sum6) or 0, 1, 2, 4, 5, 6 (FP64:
    // halving_sum6) of the group hold the sums of DOFs 0..5; the other lanes mirror DOF 0 and store
    // nothing
    const int slot6 = sub >= 8 ? -1 : kMixed ? (sub < 6 ? sub : -1) : halving_slot6(sub);
    const bool act = valid && slot6 >= 0;
    const int d = slot6 >= 0 ? slot6 : 0;
    const int64_t pc_ = valid ? p : 0;
    int r0 = 0, r1 = 0;
    if (valid) {
        r0 = m.row[p];
        r1 = m.row[p + 1];
    }
    // ---- the particle's own records (step mode), issued ahead of the gather
    double *ps = m.pstate + 16 * pc_;
    double *pd = m.pdyn + 8 * pc_;
    const double *pc = m.pconst + 8 * pc_;
    const bool has_fext = m.f_ext != nullptr;
    double im = 0.0, vh = 0.0, q0 = 0.0, fa_old = 0.0, fe = 0.0;
    int mask = 0, sp = 0;
    if (MODE != GATHER_ASSEMBLE) {
        im = pc[d];
        mask = (int)(((uint64_t)__double_as_longlong(pc[6]) >> (8 * d)) & 0xffu);
        sp = (int)__double_as_longlong(pc[7]);
        vh = ps[9 + d];
        q0 = ps[3 + d];
        if (has_fext) fe = m.f_ext[6 * pc_ + d];
    }
    // Each CSR entry is one (tetrahedron, vertex) slot: 6 values, force (3) and moment about the
    // particle (3).  Lane `sub` sums entries sub, sub + LPP, sub + 2 LPP, ... of the particle's row in
    // that order: the first kSlotTab from the slot table (all of them in flight at once, addressed by
    // the particle index alone), the rest of a longer row through row/ent.
    constexpr int KT = (kSlotTab + LPP - 1) / LPP;  // table positions per lane
    const int32_t *__restrict__ tab = m.stab + (int64_t)pc_ * kSlotTab;
    auto slot_id = [&](int k) -> int {
        const int j = sub + LPP * k;
        return (valid && j < kSlotTab) ? __ldg(tab + j) : -1;
    };
    const int j_over = sub + LPP * ((kSlotTab - sub + LPP - 1) / LPP);  // this lane's first entry past the table
    double fa_new;
    ff fa_ff{};  // mixed: the same sum as a float-float
    if constexpr (kMixed) {
        // components (0, 1), (2, 3), (4, 5) as packed float-float pairs
        ff2 a[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) a[c] = ff2{make_float2(0.0f, 0.0f), make_float2(0.0f, 0.0f)};
        {
            int id[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) id[k] = slot_id(k);
            // the shares in batches of KB entries in flight (all ids are loaded above): 48 registers,
            // 20 blocks of 64 threads per SM
            constexpr int KB = 2;
#pragma unroll
            for (int k0 = 0; k0 < KT; k0 += KB) {
                float2 w[KB][3];
#pragma unroll
                for (int k = k0; k < k0 + KB && k < KT; ++k)
                    if (id[k] >= 0) {
                        const float2 *src = reinterpret_cast<const float2 *>(tvc + 6 * (int64_t)id[k]);
                        w[k - k0][0] = ld_live<PERSIST>(src);
                        w[k - k0][1] = ld_live<PERSIST>(src + 1);
                        w[k - k0][2] = ld_live<PERSIST>(src + 2);
                    }
#pragma unroll
                for (int k = k0; k < k0 + KB && k < KT; ++k)
                    if (id[k] >= 0) {
#pragma unroll
                        for (int c = 0; c < 3; ++c) ff2_acc(a[c], w[k - k0][c]);
                    }
            }
        }
        for (int j = j_over; j < r1 - r0; j += LPP) {  // rows longer than the table
            const float2 *src = reinterpret_cast<const float2 *>(tvc + 6 * (int64_t)ent[r0 + j]);
#pragma unroll
            for (int c = 0; c < 3; ++c) ff2_acc(a[c], ld_live<PERSIST>(src + c));
        }
        // lanes beyond the first 8 of a group fold into them
#pragma unroll
        for (int off = LPP / 2; off >= 8; off >>= 1)
#pragma unroll
            for (int c = 0; c < 3; ++c) a[c] = ff2_add(a[c], ff2_shfl_xor(a[c], off));
        if (MODE != GATHER_ASSEMBLE) fa_old = pd[d];  // f_n: needed only by the energy increments
        fa_ff = ff_norm(pair_halving_sum6(a, lane));
        fa_new = ff_to_double(fa_ff);
    } else {
        double a[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) a[k] = 0.0;
        {
            int id[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) id[k] = slot_id(k);
            double2 w[KT][3];
#pragma unroll
            for (int k = 0; k < KT; ++k)
                if (id[k] >= 0) {
                    const double2 *src = reinterpret_cast<const double2 *>(tvc + 6 * (int64_t)id[k]);
                    w[k][0] = ld_live<PERSIST>(src);
                    w[k][1] = ld_live<PERSIST>(src + 1);
                    w[k][2] = ld_live<PERSIST>(src + 2);
                }
#pragma unroll
            for (int k = 0; k < KT; ++k)
                if (id[k] >= 0) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        a[2 * c] += w[k][c].x;
                        a[2 * c + 1] += w[k][c].y;
                    }
                }
        }
        for (int j = j_over; j < r1 - r0; j += LPP) {  // rows longer than the table
            const double2 *src = reinterpret_cast<const double2 *>(tvc + 6 * (int64_t)ent[r0 + j]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double2 w = ld_live<PERSIST>(src + c);
                a[2 * c] += w.x;
                a[2 * c + 1] += w.y;
            }
        }
#pragma unroll
        for (int off = LPP / 2; off >= 8; off >>= 1)
#pragma unroll
            for (int k = 0; k < 6; ++k) a[k] += __shfl_xor_sync(0xffffffffu, a[k], off);
        if (MODE != GATHER_ASSEMBLE) fa_old = pd[d];
        halving_sum6(a, lane);
        fa_new = a[0];
    }
    if (MODE == GATHER_ASSEMBLE) {
        if (act) out6[6 * p + d] = fa_new;
        return;
    }
    // ---- velocity-form central difference for DOF d (state on entry: q_{n+1}, v_{n+1/2}, f_n)
    const SpecDyn &S = m.spec[sp];
    const double dt = S.dt, hdt = S.half_dt;
    // energy terms need the external work only where a lane is constrained or loaded
    const bool need_we = __any_sync(0xffffffffu, act && (mask != 0 || has_fext));
    // prescribed velocity vb ramp(t): the constraint's accelerations at t_n and t_{n+1} are
    // vb (ramp(t +- dt/2) differences) / dt, so their sum telescopes to vb (r(t1+dt/2) - r(t0-dt/2)) / dt
    double g_bc = 0.0, v_bc = 0.0;
    if (mask > 1) {
        const int64_t n1 = ld_live<PERSIST>(reinterpret_cast<const long long *>(m.step));
        const double t1 = (double)n1 * dt;
        const double r_next = ramp(t1 + hdt, S.inv_ramp);
        g_bc = m.bc_vm[6 * pc_ + d] * (r_next - ramp(t1 - dt - hdt, S.inv_ramp)) * S.inv_dt;
        v_bc = m.bc_vel[6 * pc_ + d] * r_next;
    }
    double v_next, dWi_acc, dWe_acc;
    if (mask == 0) {
        const double fa = has_fext ? fe + fa_new : fa_new;
        if constexpr (kMixed) {
            v_next = fma(fa, dt * im, vh);  // v_{n+3/2} = v_{n+1/2} + dt a_{n+1}
        } else {
            const double dv = fa * (hdt * im);  // dt/2 a_{n+1}
            v_next = (vh + dv) + dv;
        }
    } else {
        v_next = mask == 1 ? 0.0 : v_bc;
    }
    // energy increments over [t_n, t_{n+1}] (trapezoid): dq = dt v_{n+1/2},
    //   dW_int = -(f_n + f_{n+1}) dq / 2 on every DOF, dW_ext = g dq / 2 with g the sum of the
    //   external forces (2 f_ext on loaded DOFs, the supports' reactions on constrained ones)
    if constexpr (kMixed) {
        // float-float products with v_{n+1/2}, summed over the six DOFs as one packed pair
        // (internal, external); the common factor dt/2 is applied in FP64 when accumulating
        const ff fsum = ff_add(ff_from_double(fa_old), fa_ff);
        const ff vhf = ff_from_double(vh);
        ff g = {0.0f, 0.0f};
        if (mask == 0) {
            if (has_fext) {
                const ff f1 = ff_from_double(fe);
                g = ff{2.0f * f1.hi, 2.0f * f1.lo};
            }
        } else {
            g = mask == 1 ? ff_neg(fsum) : ff_add(ff_from_double(g_bc), ff_neg(fsum));
        }
        const ff zero = {0.0f, 0.0f};
        ff2 e = ff2_pack(act ? ff_neg(ff_mul(fsum, vhf)) : zero, (need_we && act) ? ff_mul(g, vhf) : zero);
        // the six DOF contributions into every lane of the group (lanes 6, 7 hold zeros)
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) e = ff2_add(e, ff2_shfl_xor(e, off));
        dWi_acc = f2d_bits(e.hi.x) + f2d_bits(e.lo.x);
        dWe_acc = need_we ? f2d_bits(e.hi.y) + f2d_bits(e.lo.y) : 0.0;
    } else {
        double g_sum = 0.0;
        if (mask == 0) {
            if (has_fext) g_sum = 2.0 * fe;
        } else if (mask == 1) {
            g_sum = -(fa_old + fa_new);
        } else {
            g_sum = g_bc - (fa_old + fa_new);
        }
        const double hdq = hdt * vh;
        double dWi = act ? -(fa_old + fa_new) * hdq : 0.0;
        double dWe = (need_we && act) ? g_sum * hdq : 0.0;
        // sum the six DOF contributions into lane 0 of the group (lanes 3, 7 hold zeros)
#pragma unroll
        for (int off = 4; off > 0; off >>= 1) dWi += __shfl_xor_sync(0xffffffffu, dWi, off);
        if (need_we) {
#pragma unroll
            for (int off = 4; off > 0; off >>= 1) dWe += __shfl_xor_sync(0xffffffffu, dWe, off);
        }
        dWi_acc = dWi;
        dWe_acc = dWe;
    }
    // store the drifted state of the next step: v_{n+3/2} and q_{n+2} = q_{n+1} + dt v_{n+3/2}
    const double q = q0 + dt * v_next;
    if (act) {
        pd[d] = fa_new;
        ps[3 + d] = q;
        ps[9 + d] = v_next;
        if (m.pm32) write_mirror(m.pm32 + kMirror * pc_, d, q, v_next);
        if (!finite_bits(v_next) || !finite_bits(q)) *(volatile int32_t *)m.flag = 1;
        if (sub == 0) {
            if constexpr (kMixed) {
                pd[6] = fma(hdt, dWi_acc, pd[6]);
                if (need_we) pd[7] = fma(hdt, dWe_acc, pd[7]);
            } else {
                pd[6] += dWi_acc;
                if (need_we) pd[7] += dWe_acc;
            }
        }
    }
}

template <class R, int MODE, int LPP>
__global__ void __launch_bounds__(64, sizeof(R) == 4 ? 20 : 1) gather_kernel(DeviceModel m, double *__restrict__ out6)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * (32 / LPP) + lane / LPP;
    gather_group<R, MODE, LPP, false>(m, p, lane, out6);
}

// ------------------------------------------------------------------------------------------------
// Persistent step kernel: one cooperative launch runs `nsteps` whole steps.  Each step is the facet
// pass (warps take 8-tetrahedron tiles in a grid-stride loop), a grid barrier, the particle pass (warps
// take groups of 4 particles), and a second grid barrier; the arithmetic and summation orders are
// those of facet_warp_kernel and gather_kernel<.., 8>, so results equal the launch-pair path bit for
// bit.  The cooperative launch guarantees that all blocks are resident, so every barrier completes
// unless a block fails to arrive; each wait is nevertheless bounded (PersistCtl::wait_ns of
// %globaltimer and kMaxPolls polls), after which the block sets the status word and returns, and
// every other block stops at its next wait.
// ------------------------------------------------------------------------------------------------
constexpr uint32_t kMaxPolls = 1u << 24;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Strong relaxed load at GPU scope: served by L2, and, unlike an acquire, it does not invalidate the
// SM's L1 at every poll (which would cost the blocks still working on that SM their cached lines).
__device__ __forceinline__ unsigned ld_relaxed_gpu(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Barrier `target / gridDim.x` of the launch: all blocks' writes before it are visible to all blocks
// after it.  After the block's __syncthreads, thread 0 arrives with a release reduction on the
// arrival counter (it orders the block's earlier writes before the arrival; with `arrive` false, the
// fault-injection hook, it does not arrive) and polls the count with relaxed loads, spinning for 256
// polls and then sleeping 64 ns between polls, until it reaches `target`; an acquire fence after the
// last poll then orders the other blocks' writes before the block's later reads (a relaxed read
// followed by a fence is an acquire in the PTX memory model).  Returns false in every thread of the
// block if the wait gave up: its own limit was reached (the status word is set), or another block had
// set the status.
__device__ __forceinline__ bool grid_barrier(const PersistCtl &c, unsigned target, bool arrive)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        if (arrive) asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(c.arrive) : "memory");
        const uint64_t t0 = global_ns();
        for (uint32_t it = 0;; ++it) {
            if (ld_relaxed_gpu(c.arrive) >= target) break;
            if (*(volatile const int32_t *)c.status != 0) {
                ok = 0;
                break;
            }
            if (it >= kMaxPolls || global_ns() - t0 > c.wait_ns) {
                atomicCAS(c.status, 0, kStatusTimeout);
                ok = 0;
                break;
            }
            if (it > 256) __nanosleep(64);
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

template <class R, bool PF, bool S1, int WPB>
__global__ void __launch_bounds__(32 * WPB)
    step_persistent_kernel(const __grid_constant__ DeviceModel m, const void *__restrict__ vsrc, int64_t nsteps,
                           PersistCtl ctl)
{
    constexpr int TETS = kTileTets;
    __shared__ alignas(16) R sv_[WPB][TETS * 4][Stride<R>::row];
    __shared__ alignas(16) R spl_[WPB][6 * kPlane];
    __shared__ R seV_[WPB][TETS];
    __shared__ int sok_[WPB][TETS];
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = *(volatile const int32_t *)ctl.status;
    __syncthreads();
    if (s_stop != 0) return;  // an earlier launch gave up: no work (the whole block)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * WPB + w, nw = (int64_t)gridDim.x * WPB;
    const int64_t tiles = m.T / TETS;             // T is a multiple of the tile
    const int64_t groups = ((int64_t)m.N + 3) / 4;  // 4 particles of 8 lanes per warp
    unsigned target = 0;
    for (int64_t n = 0; n < nsteps; ++n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *m.step += 1;
        for (int64_t t = gw; t < tiles; t += nw)
            facet_tile<R, FACET_STEP, PF, S1, true>(m, vsrc, t * TETS, lane, sv_[w], spl_[w], seV_[w], sok_[w]);
        target += gridDim.x;
        if (!grid_barrier(ctl, target, !(n == 0 && (int)blockIdx.x == ctl.skip_block))) return;
        for (int64_t g = gw; g < groups; g += nw) gather_group<R, GATHER_STEP_MID, 8, true>(m, 4 * g + lane / 8, lane, nullptr);
        target += gridDim.x;
        if (!grid_barrier(ctl, target, true)) return;
    }
}

// FP64 variant: the facet phase takes 8-tetrahedron tiles per block of 96 threads, one facet per thread
// (facet_block_tile, as facet_kernel does), which gives the FP64 pipe 4x the warps of warp tiles with
// three facets per lane.  The particle phase is the warp-level one of the kernel above.
template <class R, bool PF>
__global__ void __launch_bounds__(12 * kTileTets)
    step_persistent_block_kernel(const __grid_constant__ DeviceModel m, const void *__restrict__ vsrc, int64_t nsteps,
                                 PersistCtl ctl)
{
    constexpr int TETS = kTileTets;
    constexpr int WPB = 12 * TETS / 32;
    __shared__ alignas(16) R sv[TETS * 4][Stride<R>::row];
    __shared__ alignas(16) R scon[12 * TETS][Stride<R>::con];
    __shared__ R seV[TETS];
    __shared__ int sok[TETS];
    __shared__ int s_stop;
    if (threadIdx.x == 0) s_stop = *(volatile const int32_t *)ctl.status;
    __syncthreads();
    if (s_stop != 0) return;  // an earlier launch gave up: no work (the whole block)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t gw = (int64_t)blockIdx.x * WPB + w, nw = (int64_t)gridDim.x * WPB;
    const int64_t tiles = m.T / TETS;
    const int64_t groups = ((int64_t)m.N + 3) / 4;
    unsigned target = 0;
    for (int64_t n = 0; n < nsteps; ++n) {
        if (blockIdx.x == 0 && threadIdx.x == 0) *m.step += 1;
        for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x)
            facet_block_tile<R, FACET_STEP, TETS, PF, true>(m, vsrc, t * TETS, sv, scon, seV, sok);
        target += gridDim.x;
        if (!grid_barrier(ctl, target, !(n == 0 && (int)blockIdx.x == ctl.skip_block))) return;
        for (int64_t g = gw; g < groups; g += nw) gather_group<R, GATHER_STEP_MID, 8, true>(m, 4 * g + lane / 8, lane, nullptr);
        target += gridDim.x;
        if (!grid_barrier(ctl, target, true)) return;
    }
}

template <class R, bool PF, bool S1>
constexpr int persist_wpb()
{
    return sizeof(R) == 4 ? 4 : 12 * kTileTets / 32;  // static shared memory stays below 48 KB per block
}

template <class R, bool PF, bool S1>
const void *persist_fn()
{
    if constexpr (sizeof(R) == 4)
        return reinterpret_cast<const void *>(&step_persistent_kernel<R, PF, S1, persist_wpb<R, PF, S1>()>);
    else
        return reinterpret_cast<const void *>(&step_persistent_block_kernel<R, PF>);
}

// First half kick and drift of a stepping call: v_{n+1/2} = v_n + dt/2 a_n, q_{n+1} = q_n + dt v_{n+1/2}.
__global__ void __launch_bounds__(256) kick_kernel(DeviceModel m)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * (int64_t)m.N) return;
    const int64_t p = i / 6;
    const int d = (int)(i - 6 * p);
    double *ps = m.pstate + 16 * p;
    const double *pc = m.pconst + 8 * p;
    const int mask = (int)(((uint64_t)__double_as_longlong(pc[6]) >> (8 * d)) & 0xffu);
    const int sp = (int)__double_as_longlong(pc[7]);
    const double dt = m.spec[sp].dt;
    double vh;
    if (mask == 0) {
        const double fe = m.f_ext ? m.f_ext[6 * p + d] : 0.0;
        vh = ps[9 + d] + 0.5 * dt * (fe + m.pdyn[8 * p + d]) * pc[d];
    } else if (mask == 1) {
        vh = 0.0;
    } else {
        const double t = (double)(*m.step) * dt;
        vh = m.bc_vel[6 * p + d] * ramp(t + 0.5 * dt, m.spec[sp].inv_ramp);
    }
    const double q = ps[3 + d] + dt * vh;
    ps[9 + d] = vh;
    ps[3 + d] = q;
    if (m.pm32) write_mirror(m.pm32 + kMirror * p, d, q, vh);
}

// Whole-step values (q_n, v_n) of DOF d of internal particle p from the drifted state (q_{n+1},
// v_{n+1/2}) the library keeps between calls: the inverse of kick_kernel under the same boundary
// conditions.
__device__ __forceinline__ void unkick_dof(const DeviceModel &m, int64_t p, int d, double &qn, double &vn)
{
    const double *ps = m.pstate + 16 * p;
    const double *pc = m.pconst + 8 * p;
    const int mask = (int)(((uint64_t)__double_as_longlong(pc[6]) >> (8 * d)) & 0xffu);
    const SpecDyn &S = m.spec[(int)__double_as_longlong(pc[7])];
    const double vh = ps[9 + d];
    if (mask == 0) {
        const double fe = m.f_ext ? m.f_ext[6 * p + d] : 0.0;
        vn = vh - S.half_dt * (fe + m.pdyn[8 * p + d]) * pc[d];
    } else if (mask == 1) {
        vn = 0.0;
    } else {
        vn = m.bc_vel[6 * p + d] * ramp((double)(*m.step) * S.dt, S.inv_ramp);
    }
    qn = ps[3 + d] - S.dt * vh;
}

// Whole-step state into out12 [N][12] (q then v, internal order), or with out12 null into pstate (and
// the mirror) in place.
__global__ void __launch_bounds__(256) unkick_kernel(DeviceModel m, double *__restrict__ out12)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * (int64_t)m.N) return;
    const int64_t p = i / 6;
    const int d = (int)(i - 6 * p);
    double qn, vn;
    unkick_dof(m, p, d, qn, vn);
    if (out12) {
        out12[12 * p + d] = qn;
        out12[12 * p + 6 + d] = vn;
    } else {
        double *ps = m.pstate + 16 * p;
        ps[3 + d] = qn;
        ps[9 + d] = vn;
        if (m.pm32) write_mirror(m.pm32 + kMirror * p, d, qn, vn);
    }
}

// Whole-step state in the caller's particle order: caller particle k is internal particle pmap[k];
// q, v [n][6] (either may be null).
__global__ void __launch_bounds__(256) state_to_user_kernel(DeviceModel m, const int32_t *__restrict__ pmap, int64_t n,
                                                            double *__restrict__ q, double *__restrict__ v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * n) return;
    const int64_t k = i / 6;
    const int d = (int)(i - 6 * k);
    double qn, vn;
    unkick_dof(m, pmap[k], d, qn, vn);
    if (q) q[i] = qn;
    if (v) v[i] = vn;
}

// FP32 mirror of every particle from the FP64 records.
__global__ void __launch_bounds__(256) mirror_kernel(DeviceModel m)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= m.N) return;
    const double *ps = m.pstate + 16 * p;
    float *pm = m.pm32 + kMirror * p;
    for (int k = 0; k < 3; ++k) d2f_split(ps[k], pm[k], pm[3 + k]);
    for (int d = 0; d < 6; ++d) write_mirror(pm, d, ps[3 + d], ps[9 + d]);
    for (int k = 21; k < kMirror; ++k) pm[k] = 0.0f;
}

// Perturbation of the displacements and rotations of free DOFs (dq [N][6], internal order).  In the
// drifted state q_{n+1} = q_n + dt v_{n+1/2}, adding dq to q_n adds it to q_{n+1}; velocities, forces
// and history are unchanged, so the next strain increment is measured from the perturbed state.
__global__ void __launch_bounds__(256) perturb_kernel(DeviceModel m, const double *__restrict__ dq)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 6 * (int64_t)m.N) return;
    const int64_t p = i / 6;
    const int d = (int)(i - 6 * p);
    const int mask = (int)(((uint64_t)__double_as_longlong(m.pconst[8 * p + 6]) >> (8 * d)) & 0xffu);
    if (mask != 0) return;
    double *ps = m.pstate + 16 * p;
    const double q = ps[3 + d] + dq[i];
    ps[3 + d] = q;
    if (m.pm32) write_mirror(m.pm32 + kMirror * p, d, q, ps[9 + d]);
}

// Energy sums over particles [p0, p1) (per block, fixed order), then one block adds the partials.
// Warp sum of 16 values per lane by halving exchanges: at each level a lane keeps half of its values
// and adds its partner's copy of that half (8 + 4 + 2 + 1 + 1 additions).  Afterwards lanes 2i and
// 2i + 1 both hold the warp sum of value i.  The order of the additions is fixed.
__device__ __forceinline__ double warp_sum16(double (&v)[16], int lane)
{
#pragma unroll
    for (int h = 8, off = 16; h >= 1; h >>= 1, off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const double keep = upper ? v[h + i] : v[i];
            const double give = upper ? v[i] : v[h + i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, give, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

// Energy terms of particles [p0, p1): per block a fixed-order sum into partial[block][16]; the block
// that finishes last (ticket from an atomic counter that wraps back to 0) sums the partials in block
// order into out16.  No thread waits on another block.
__global__ void __launch_bounds__(256) energy_kernel(DeviceModel m, int32_t p0, int32_t p1, double *partial,
                                                     unsigned *ticket, double *out16)
{
    __shared__ double red[8][16];
    __shared__ bool last;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int64_t p = (int64_t)p0 + (int64_t)blockIdx.x * 256 + tid;
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    if (p < p1) {
        const double *ps = m.pstate + 16 * p;
        const double *pd = m.pdyn + 8 * p;
        const double *pc = m.pconst + 8 * p;
        const uint64_t bcbits = (uint64_t)__double_as_longlong(pc[6]);
        const int sp = (int)__double_as_longlong(pc[7]);
        const SpecDyn &S = m.spec[sp];
        const double dt = S.dt;
        const double t = (double)(*m.step) * dt;
        acc[0] = pd[6];
        acc[1] = pd[7];
        for (int d = 0; d < 6; ++d) {
            const double mass = 1.0 / pc[d];
            // whole-step velocity v_n from the stored v_{n+1/2} (inverse half kick)
            const int mk = (int)((bcbits >> (8 * d)) & 0xffu);
            double v = ps[9 + d];
            if (mk == 0)
                v -= S.half_dt * ((m.f_ext ? m.f_ext[6 * p + d] : 0.0) + pd[d]) * pc[d];
            else if (mk == 1)
                v = 0.0;
            else
                v = m.bc_vel[6 * p + d] * ramp(t, S.inv_ramp);
            acc[2] += 0.5 * mass * v * v;
            if (mk == 1) {
                acc[4 + d] += -pd[d];
            } else if (mk == 2) {
                const double ra = ramp(t + 0.5 * dt, S.inv_ramp) - ramp(t - 0.5 * dt, S.inv_ramp);
                acc[10 + d] += m.bc_vm[6 * p + d] * ra * S.inv_dt - pd[d];
            }
        }
    }
    const double ws = warp_sum16(acc, lane);
    if ((lane & 1) == 0) red[w][lane >> 1] = ws;
    __syncthreads();
    if (tid < 16) {
        double b = 0.0;
#pragma unroll
        for (int k = 0; k < 8; ++k) b += red[k][tid];
        partial[16 * (int64_t)blockIdx.x + tid] = b;
        __threadfence();
    }
    __syncthreads();
    if (tid == 0) last = atomicInc(ticket, gridDim.x - 1) == gridDim.x - 1;
    __syncthreads();
    if (last && tid < 16) {
        double s = 0.0;
        for (unsigned k = 0; k < gridDim.x; ++k) s += __ldcg(partial + 16 * (int64_t)k + tid);
        out16[tid] = s;
    }
}

// History <-> caller format (t_N, global tangential traction, e_max), in the internal facet order.
// The frame is rebuilt from the particle positions exactly as the facet pass forms it.
template <class R>
__device__ __forceinline__ bool facet_frame_of(const DeviceModel &m, int64_t f, V3<R> &n, V3<R> &mt, V3<R> &lt)
{
    const int64_t tt = f / 12;
    const int e = (int)(f - 12 * tt) >> 1;
    const int va = (0x211000 >> (4 * e)) & 0xF;
    const int vb = (0x332321 >> (4 * e)) & 0xF;
    const int *tv = reinterpret_cast<const int *>(m.tet) + 4 * tt;
    const int p0 = tv[0], pa = tv[va], pb = tv[vb];
    if (p0 < 0) return false;
    V3<R> dxa, dxb;
    if constexpr (sizeof(R) == 4) {
        const float *x0 = m.pm32 + kMirror * (int64_t)p0, *xa = m.pm32 + kMirror * (int64_t)pa,
                    *xb = m.pm32 + kMirror * (int64_t)pb;
        dxa = {(xa[0] - x0[0]) + (xa[3] - x0[3]), (xa[1] - x0[1]) + (xa[4] - x0[4]),
               (xa[2] - x0[2]) + (xa[5] - x0[5])};
        dxb = {(xb[0] - x0[0]) + (xb[3] - x0[3]), (xb[1] - x0[1]) + (xb[4] - x0[4]),
               (xb[2] - x0[2]) + (xb[5] - x0[5])};
    } else {
        const double *x0 = m.pstate + 16 * (int64_t)p0, *xa = m.pstate + 16 * (int64_t)pa,
                     *xb = m.pstate + 16 * (int64_t)pb;
        dxa = {R(xa[0] - x0[0]), R(xa[1] - x0[1]), R(xa[2] - x0[2])};
        dxb = {R(xb[0] - x0[0]), R(xb[1] - x0[1]), R(xb[2] - x0[2])};
    }
    const V3<R> d = dxb - dxa;
    const R inv_l = rsqrt_(dot(d, d));
    n = inv_l * d;
    tangent_frame(n, mt, lt);
    return true;
}

// History of n facets in the caller's order: umap[k] = 2 f + s for internal facet f, s = 1 where the
// caller's facet runs from the internal vertex b to a (the tangential traction vector flips sign).
template <class R>
__global__ void hist_to_user_kernel(DeviceModel m, const int32_t *__restrict__ umap, int64_t nf,
                                    double *__restrict__ out5)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nf) return;
    const int32_t code = umap[k];
    const int64_t f = code >> 1;
    const double sg = (code & 1) ? -1.0 : 1.0;
    V3<R> n, mt, lt;
    const R4<R> h = static_cast<const R4<R> *>(m.hist)[f];
    double *o = out5 + 5 * k;
    if (!facet_frame_of<R>(m, f, n, mt, lt)) {
        for (int c = 0; c < 5; ++c) o[c] = 0.0;
        return;
    }
    o[0] = double(h.x);
    o[1] = sg * (double(h.y) * double(mt.x) + double(h.z) * double(lt.x));
    o[2] = sg * (double(h.y) * double(mt.y) + double(h.z) * double(lt.y));
    o[3] = sg * (double(h.y) * double(mt.z) + double(h.z) * double(lt.z));
    o[4] = double(h.w);
}

template <class R>
__global__ void hist_from_user_kernel(DeviceModel m, const double *__restrict__ in5)
{
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= 12 * (int64_t)m.T) return;
    V3<R> n, mt, lt;
    R4<R> h;
    h.x = h.y = h.z = h.w = R(0);
    if (facet_frame_of<R>(m, f, n, mt, lt)) {
        const double *u = in5 + 5 * f;
        h.x = R(u[0]);
        h.y = R(u[1] * double(mt.x) + u[2] * double(mt.y) + u[3] * double(mt.z));
        h.z = R(u[1] * double(lt.x) + u[2] * double(lt.y) + u[3] * double(lt.z));
        h.w = R(u[4]);
    }
    static_cast<R4<R> *>(m.hist)[f] = h;
}

template <class R, int MODE, bool PF>
cudaError_t launch_facet_pf(const DeviceModel &m, const void *pst, cudaStream_t s, const BatchLaw *bl)
{
    const int tpb = m.tets_per_block;
    const unsigned blocks = (unsigned)((m.T + tpb - 1) / tpb);
    if (blocks == 0) return cudaSuccess;
    // FP32 facet pass with 8-tetrahedron tiles: one tile per warp, 2 warps per block (measured on GB300:
    // 43.6 us against 47.4 us for the 96-thread block kernel on 1.82M facets).  The FP64 pass, bound by
    // the FP64 pipe, is 4 % faster with the block kernel.
    if (sizeof(R) == 4 && tpb == kTileTets) {
        constexpr int WPB = 2;
        const int64_t tiles = (m.T + kTileTets - 1) / kTileTets;
        const unsigned nb = (unsigned)((tiles + WPB - 1) / WPB);
        if (m.n_spec == 1)
            facet_warp_kernel<R, MODE, WPB, PF, true><<<nb, 32 * WPB, 0, s>>>(m, pst);
        else if (bl && bl->n == m.n_spec)
            facet_warp_batch_kernel<MODE, WPB, PF><<<nb, 32 * WPB, 0, s>>>(m, pst, *bl);
        else
            facet_warp_kernel<R, MODE, WPB, PF, false><<<nb, 32 * WPB, 0, s>>>(m, pst);
        return cudaGetLastError();
    }
    switch (tpb) {
    case 16:
        facet_kernel<R, MODE, 16, PF><<<blocks, 192, 0, s>>>(m, pst);
        break;
    case 32:
        facet_kernel<R, MODE, 32, PF><<<blocks, 384, 0, s>>>(m, pst);
        break;
    default:
        facet_kernel<R, MODE, 8, PF><<<blocks, 96, 0, s>>>(m, pst);
        break;
    }
    return cudaGetLastError();
}

// Per-facet parameters matter only where the law or E0 / alpha enter: the step and the metrics.
template <class R, int MODE>
cudaError_t launch_facet_tpb(const DeviceModel &m, const void *pst, cudaStream_t s, const BatchLaw *bl)
{
    if constexpr (MODE == FACET_STEP || MODE == FACET_METRIC)
        if (m.pf) return launch_facet_pf<R, MODE, true>(m, pst, s, bl);
    return launch_facet_pf<R, MODE, false>(m, pst, s, bl);
}

// Persistent launch of `nsteps` steps (cooperative; grid = resident blocks per SM x SMs).  Returns
// cudaErrorCooperativeLaunchTooLarge (or another launch error) if the grid cannot be co-resident.
template <class R>
cudaError_t launch_persistent_r(const DeviceModel &m, int64_t nsteps, const PersistCtl &ctl, int *grid_out,
                                cudaStream_t s)
{
    const void *fn = (sizeof(R) == 4 && m.n_spec == 1) ? (m.pf ? persist_fn<R, true, true>() : persist_fn<R, false, true>())
                                                        : (m.pf ? persist_fn<R, true, false>() : persist_fn<R, false, false>());
    const int threads = 32 * persist_wpb<R, false, false>();
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    // as many blocks as the device holds at once, but no more than the work needs: every block takes
    // part in every barrier, so idle blocks on a small specimen would only slow the barriers down
    // (a tile takes a warp in the FP32 kernel and a block in the FP64 one; 4 particles take a warp)
    const int wpb = threads / 32;
    const int64_t tiles = m.T / kTileTets, groups = ((int64_t)m.N + 3) / 4;
    const int64_t need = sizeof(R) == 4 ? (std::max(tiles, groups) + wpb - 1) / wpb
                                        : std::max(tiles, (groups + wpb - 1) / wpb);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, need));
    if (grid_out) *grid_out = (int)grid;
    if (nsteps <= 0) return cudaSuccess;
    const void *vsrc = sizeof(R) == 4 ? static_cast<const void *>(m.pm32) : static_cast<const void *>(m.pstate);
    DeviceModel mm = m;
    int64_t ns = nsteps;
    PersistCtl c = ctl;
    void *args[] = {&mm, &vsrc, &ns, &c};
    e = cudaMemsetAsync(ctl.arrive, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return e;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(threads), args, 0, s);
}

}  // namespace

cudaError_t launch_unkick(const DeviceModel &m, double *out12, cudaStream_t s)
{
    const int64_t n = 6 * (int64_t)m.N;
    if (n == 0) return cudaSuccess;
    unkick_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, out12);
    return cudaGetLastError();
}

cudaError_t launch_state_to_user(const DeviceModel &m, const int32_t *pmap, int64_t n, double *q, double *v,
                                 cudaStream_t s)
{
    if (n <= 0 || (!q && !v)) return cudaSuccess;
    state_to_user_kernel<<<(unsigned)((6 * n + 255) / 256), 256, 0, s>>>(m, pmap, n, q, v);
    return cudaGetLastError();
}

cudaError_t launch_kick(const DeviceModel &m, cudaStream_t s)
{
    const int64_t n = 6 * (int64_t)m.N;
    if (n == 0) return cudaSuccess;
    kick_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_facet(const DeviceModel &m, int mode, const void *src_override, cudaStream_t s,
                         const BatchLaw *bl)
{
    const void *pst = src_override ? src_override
                                   : (sizeof(R) == 4 ? static_cast<const void *>(m.pm32)
                                                     : static_cast<const void *>(m.pstate));
    switch (mode) {
    case FACET_FROM_HIST:
        return launch_facet_tpb<R, FACET_FROM_HIST>(m, pst, s, bl);
    case FACET_ELASTIC:
        return launch_facet_tpb<R, FACET_ELASTIC>(m, pst, s, bl);
    case FACET_METRIC:
        return launch_facet_tpb<R, FACET_METRIC>(m, pst, s, bl);
    default:
        return launch_facet_tpb<R, FACET_STEP>(m, pst, s, bl);
    }
}

template <class R, int LPP>
cudaError_t launch_gather_lpp(const DeviceModel &m, int mode, double *out6, cudaStream_t s)
{
    const int64_t warps = ((int64_t)m.N + (32 / LPP) - 1) / (32 / LPP);
    // blocks of 2 warps, up to 20 per SM at 48 registers (mixed mode; measured on GB300 against 12, 16
    // and 18 per SM with more shares in flight, and against 8-warp blocks)
    const unsigned blocks = (unsigned)((warps * 32 + 63) / 64);
    switch (mode) {
    case GATHER_ASSEMBLE:
        gather_kernel<R, GATHER_ASSEMBLE, LPP><<<blocks, 64, 0, s>>>(m, out6);
        break;
    default:
        gather_kernel<R, GATHER_STEP_MID, LPP><<<blocks, 64, 0, s>>>(m, out6);
        break;
    }
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_gather(const DeviceModel &m, int mode, double *out6, cudaStream_t s)
{
    if (m.N == 0) return cudaSuccess;
    switch (m.gather_lanes) {
    case 32:
        return launch_gather_lpp<R, 32>(m, mode, out6, s);
    case 16:
        return launch_gather_lpp<R, 16>(m, mode, out6, s);
    default:
        return launch_gather_lpp<R, 8>(m, mode, out6, s);
    }
}

cudaError_t launch_mirror(const DeviceModel &m, cudaStream_t s)
{
    if (!m.pm32 || m.N == 0) return cudaSuccess;
    mirror_kernel<<<(unsigned)((m.N + 255) / 256), 256, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t launch_perturb(const DeviceModel &m, const double *dq, cudaStream_t s)
{
    const int64_t n = 6 * (int64_t)m.N;
    if (n == 0) return cudaSuccess;
    perturb_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, dq);
    return cudaGetLastError();
}

cudaError_t launch_energy(const DeviceModel &m, int32_t p0, int32_t p1, double *partial, unsigned *ticket,
                          double *out16, cudaStream_t s)
{
    const int32_t nb = (p1 - p0 + 255) / 256;
    if (nb <= 0) return cudaMemsetAsync(out16, 0, 16 * sizeof(double), s);
    energy_kernel<<<nb, 256, 0, s>>>(m, p0, p1, partial, ticket, out16);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_hist_to_user(const DeviceModel &m, const int32_t *umap, int64_t n, double *out5, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    hist_to_user_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, umap, n, out5);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_hist_from_user(const DeviceModel &m, const double *in5, cudaStream_t s)
{
    const int64_t n = 12 * (int64_t)m.T;
    if (n == 0) return cudaSuccess;
    hist_from_user_kernel<R><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m, in5);
    return cudaGetLastError();
}

template <class R>
cudaError_t launch_persistent(const DeviceModel &m, int64_t nsteps, const PersistCtl &ctl, int *grid_out,
                              cudaStream_t s)
{
    return launch_persistent_r<R>(m, nsteps, ctl, grid_out, s);
}

template cudaError_t launch_persistent<float>(const DeviceModel &, int64_t, const PersistCtl &, int *, cudaStream_t);
template cudaError_t launch_persistent<double>(const DeviceModel &, int64_t, const PersistCtl &, int *, cudaStream_t);
template cudaError_t launch_facet<float>(const DeviceModel &, int, const void *, cudaStream_t, const BatchLaw *);
template cudaError_t launch_facet<double>(const DeviceModel &, int, const void *, cudaStream_t, const BatchLaw *);
template cudaError_t launch_gather<float>(const DeviceModel &, int, double *, cudaStream_t);
template cudaError_t launch_gather<double>(const DeviceModel &, int, double *, cudaStream_t);
template cudaError_t launch_hist_to_user<float>(const DeviceModel &, const int32_t *, int64_t, double *, cudaStream_t);
template cudaError_t launch_hist_to_user<double>(const DeviceModel &, const int32_t *, int64_t, double *, cudaStream_t);
template cudaError_t launch_hist_from_user<float>(const DeviceModel &, const double *, cudaStream_t);
template cudaError_t launch_hist_from_user<double>(const DeviceModel &, const double *, cudaStream_t);

}  // namespace ldpm
