// ldpm_internal.h -- layouts and launcher declarations shared by the host runtime (ldpm_api.cu)
// and the kernels (ldpm_kernels.cu).  Not part of the public ABI.
//
// Device layout (all arrays in the library's internal order: particles and tetrahedra sorted along a
// Morton curve, facets tetrahedron-major with 12 consecutive slots per tetrahedron):
//   pstate [N][16] f64  x(3) q(6) v(6) pad      gathered by the facet pass (one 128-byte line);
//                       between calls q = q_{n+1} and v = v_{n+1/2} (drifted state of step n)
//   pdyn   [N][8]  f64  f_asm(6) W_int W_ext     node force sums of the current step, energy sums
//   pconst [N][8]  f64  1/mass(6) bc-bits spec   per-DOF inverse mass, 8-bit BC code per DOF, specimen
//   pm32   [N][24] f32  mixed mode only: FP32 mirror read by the facet pass, written by the particle
//                       kernels: x_hi(3) x_lo(3) u_hi(3) u_lo(3) theta(3) v(3) omega(3) pad(3), where
//                       hi = float(a), lo = float(a - hi) (a two-float split of an FP64 value)
//   tet    [T]     int4 particle ids of the 4 vertices (-1: padding tetrahedron)
//   geo    [12T]   R4   c_a (arm from the edge's first vertex to the facet centroid), projected area A
//   hist   [12T]   R4   t_N, t_M, t_L, e_max
//   pf     [12T]   R4   optional per-facet E0, alpha, sigma_t, 0 (null: the material's values)
//   fout   [12T]   R4   facet force acting on the edge's first vertex, 0 (written only when forces
//                       are rebuilt from history, for ldpm_facet_forces)
//   tvc    [T][4][6] R  per tetrahedron vertex: sum of its 6 facets' force (3) and moment about the
//                       vertex (3), in a fixed order
//   row    [N+1]   i32  CSR of (tetrahedron, vertex) slots per particle, ascending tetrahedron
//   ent    [4T]    i32  slot id 4 * tet + vertex
//   stab   [N][40] i32  the first kSlotTab entries of each particle's CSR row, -1 after its last
//                       entry: the particle pass reads a particle's slot ids from its index alone
//                       (the rest of a longer row is read through row/ent)
// Facet slot s of a tetrahedron belongs to edge e = s / 2 with local vertices
// (a, b) in ((0,1),(0,2),(0,3),(1,2),(1,3),(2,3)); "I" of the internal facet is vertex a.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ldpm {

constexpr int kMirror = 24;  // floats per particle in the FP32 mirror
constexpr int kSlotTab = 40; // slot ids per particle in stab (a multiple of 8 lanes)

struct alignas(32) double4a {
    double x, y, z, w;
};

template <class R>
struct Vec4;
template <>
struct Vec4<float> {
    using type = float4;
};
template <>
struct Vec4<double> {
    using type = double4a;
};
template <class R>
using R4 = typename Vec4<R>::type;

// Constants of the facet law in the facet pass's precision, derived once on the host.
template <class R>
struct LawConst {
    R E0, alpha, inv_alpha, sigma_t, four_alpha_over_r2, Hs_over_alpha, n_t, l_t;
    R sigma_c0, Hc0, Hc1, kc1, kc2, ec0, ec1, eV0, beta, Ed;
    R mu_diff_sN0, mu_inf, inv_sigma_N0, sigma_s;
    R dt;
    R tiny_strain;  // fracture branch: effective strains below this respond elastically
    // ratios from which the constants above that depend on E0, alpha, sigma_t are rebuilt per facet
    // (facet_params): 4 / r_st^2, r_st, H_c0/E0, H_c1/E0, kappa_c0, kappa_c3, E_d/E0
    R four_over_r2, r_st, Hc0_E0, Hc1_E0, kc0, kc3, Ed_E0, r_s;
    R k_t;  // tensile reload: traction stays zero up to e_tr = k_t (e_max - sigma_bt / E0)
    int32_t elastic;
};

// Law constants of a batch of up to kParamSpecimens specimens for the kernel parameters of the FP32
// facet pass (the copy in `law` serves larger batches).  A facet-pass block of 16 tetrahedra never
// straddles two specimens (each is padded to 32), so a block finds its specimen from t0.
constexpr int kParamSpecimens = 64;
struct BatchLaw {
    int32_t n = 0;                     // specimens; 0: not in use
    int32_t t0[kParamSpecimens + 1];   // first internal tetrahedron of each specimen, t0[n] = T
    LawConst<float> law[kParamSpecimens];
};

// Per-specimen time integration constants (FP64).
struct SpecDyn {
    double dt, ramp_time;
    double inv_dt, inv_ramp;  // 1/dt; 1/ramp_time (0 when ramp_time <= 0: no ramp)
    double half_dt;
};

// FACET_METRIC: crack opening and tetrahedron volumetric strain of the whole-step state, written to
// fout (.x = w per facet, .y = e_V of the facet's tetrahedron); history unchanged.
enum FacetMode : int { FACET_STEP = 0, FACET_FROM_HIST = 1, FACET_ELASTIC = 2, FACET_METRIC = 3 };
enum GatherMode : int { GATHER_ASSEMBLE = 0, GATHER_STEP_MID = 1 };

struct DeviceModel {
    int32_t N = 0, T = 0;     // T includes padding tetrahedra
    int32_t n_spec = 0;
    int32_t tets_per_block = 32;
    double *pstate = nullptr, *pdyn = nullptr, *pconst = nullptr;
    float *pm32 = nullptr;          // FP32 mirror (mixed mode), null in FP64 mode
    int32_t gather_lanes = 8;       // lanes per particle in the particle pass (8, 16 or 32)
    int32_t blocks_per_sm = 0;      // cap on resident facet-pass blocks per SM (0 = occupancy limit)
    double *bc_vel = nullptr, *f_ext = nullptr;
    double *bc_vm = nullptr;        // [N][6] prescribed velocity times the DOF's mass
    int4 *tet = nullptr;
    void *geo = nullptr, *hist = nullptr, *fout = nullptr, *tvc = nullptr, *ent = nullptr;
    void *hist_out = nullptr;  // where a stepping facet pass writes the new history (null: hist, in place)
    void *pf = nullptr;             // per-facet E0, alpha, sigma_t (R4 [12T]) or null
    int32_t *row = nullptr;
    int32_t *stab = nullptr;        // [N][kSlotTab] slot ids per particle (see the layout above)
    int32_t *tile_spec = nullptr;   // [T / tets_per_block] specimen of each tile, or null (all 0)
    void *law = nullptr;            // LawConst<R>[n_spec]
    LawConst<float> law1{};         // mixed mode, one specimen: lawc[0] again, read from the kernel parameters
    SpecDyn *spec = nullptr;        // [n_spec]
    int64_t *step = nullptr;        // step counter (one for all specimens)
    int32_t *flag = nullptr;        // non-finite state seen
};

// Control block of the persistent step kernel.  `arrive` counts the blocks' arrivals at the grid
// barriers of one launch (zeroed before the launch); `status` is 0, or kStatusTimeout once a barrier
// wait gave up (it stays set: later persistent launches return at once, and the handle reports
// LDPM_E_TIMEOUT until its state is replaced); `wait_ns` bounds one barrier wait; block `skip_block`
// (-1: none) does not arrive at the first barrier of the launch (fault injection for tests).
constexpr int32_t kStatusTimeout = 1;
struct PersistCtl {
    unsigned *arrive = nullptr;
    int32_t *status = nullptr;
    uint64_t wait_ns = 2000000000ull;
    int32_t skip_block = -1;
};

// Reverse (adjoint) pass workspace (ldpm_adjoint.cu).  The objective is
//   J = sum_n sum_i c_i f_i(t_n),  c = -seed / K on constrained DOFs, 0 elsewhere
// (the time mean of the seeded reactions R = m a - f), and its gradient with respect to the
// per-facet E0, alpha, sigma_t.  Reverse step n reads the inputs of forward step n: the particle
// records it read (snap_p: pm32 layout in mixed mode, pstate layout in FP64) and the history before it
// (snap_h).
//   af     [N][8] f64 (FP64) or [N][12] f32 (mixed: a_u hi(3) lo(3), a_theta(3), pad(3)):
//          a_f = c + dt M^-1 Ubar, the adjoint of the node forces of the step being reversed
//   adj_h  [12T] R4  adjoint of the history (t_N, t_M, t_L, e_max) of the step before it
//   gacc   [12T] R4  gradient accumulators (E0, alpha, sigma_t, 0)
//   tvc2   [T][4][12] R  per tetrahedron vertex: sums of the facets' displacement adjoints (6) and
//          velocity adjoints (6)
//   Qbar, Ubar [N][6] f64  adjoints of q_n and v_{n-1/2}
struct AdjointModel {
    const void *snap_p = nullptr, *snap_h = nullptr;
    void *af = nullptr, *adj_h = nullptr, *gacc = nullptr, *tvc2 = nullptr;
    double *Qbar = nullptr, *Ubar = nullptr, *cseed = nullptr;
    double *gsum = nullptr;  // [12T][4] FP64 totals (mixed mode: gacc is folded here per segment)
    double *jacc = nullptr;  // [N] per-particle shares of the objective, summed over the forward steps
    int32_t reload = 0;      // 1 if some specimen has k_t > 0 (the reload rule's derivative is needed)
};

// Message returned by ldpm_last_error() on the calling thread (ldpm_api.cu).
void set_last_error(const char *msg);

// Launchers (ldpm_kernels.cu).  All enqueue on `s` and return the launch error.
// kick: whole-step state (q_n, v_n, f_n) -> drifted state (q_{n+1}, v_{n+1/2}) kept between calls.
cudaError_t launch_kick(const DeviceModel &m, cudaStream_t s);
// unkick: the inverse; into out12 [N][12] (q_n then v_n) or, with out12 null, in place.
cudaError_t launch_unkick(const DeviceModel &m, double *out12, cudaStream_t s);
// Whole-step state in the caller's particle order: caller particle k is internal particle pmap[k];
// q, v [n][6] device arrays (either may be null).
cudaError_t launch_state_to_user(const DeviceModel &m, const int32_t *pmap, int64_t n, double *q, double *v,
                                 cudaStream_t s);
// One cooperative launch of `nsteps` steps of the persistent step kernel (mixed or FP64 by R).  The grid
// is the number of co-resident blocks (occupancy x SMs), written to *grid_out; nsteps = 0 only
// computes it.  Returns the launch error (cudaErrorCooperativeLaunchTooLarge if the grid cannot be
// resident).
template <class R>
cudaError_t launch_persistent(const DeviceModel &m, int64_t nsteps, const PersistCtl &ctl, int *grid_out,
                              cudaStream_t s);
// `src_override` replaces the particle records the facet pass reads (FP64 mode: pstate layout;
// mixed mode: pm32 layout); null = the model's own.
template <class R>
cudaError_t launch_facet(const DeviceModel &m, int mode, const void *src_override, cudaStream_t s,
                         const BatchLaw *bl = nullptr);
// q += dq on free DOFs of the drifted state (dq [N][6] internal order, device), mirror updated.
cudaError_t launch_perturb(const DeviceModel &m, const double *dq, cudaStream_t s);
// Rebuild the FP32 mirror from pstate (after create, set_state, checkpoint load).  No-op in FP64.
cudaError_t launch_mirror(const DeviceModel &m, cudaStream_t s);
template <class R>
cudaError_t launch_gather(const DeviceModel &m, int mode, double *out6, cudaStream_t s);
// Energy sums over particles [p0, p1): out16 = W_int, W_ext, W_kin, pad, reaction fixed(6),
// reaction prescribed(6).  `partial` holds ceil((p1 - p0) / 256) * 16 doubles; `ticket` is a device
// counter, 0 before the first launch, which each launch leaves at 0 again.
cudaError_t launch_energy(const DeviceModel &m, int32_t p0, int32_t p1, double *partial, unsigned *ticket,
                          double *out16, cudaStream_t s);
// History of n facets in the caller's order (out5 [n][5]: t_N, tangential traction vector, e_max);
// umap[k] = 2 f + s, f the internal facet, s = 1 where the caller's facet has the opposite orientation.
template <class R>
cudaError_t launch_hist_to_user(const DeviceModel &m, const int32_t *umap, int64_t n, double *out5, cudaStream_t s);

// Adjoint launchers (ldpm_adjoint.cu).
// Reset: af = c, Qbar = Ubar = 0, adj_h = 0, gacc = 0 (and gsum = 0).
template <class R>
cudaError_t launch_adjoint_init(const DeviceModel &m, const AdjointModel &a, cudaStream_t s);
// Reverse of one step: the facet pass (law VJP, parameter gradients, per-vertex sums), then the
// particle pass (Qbar, Ubar and the next a_f).
template <class R>
cudaError_t launch_adjoint_facet(const DeviceModel &m, const AdjointModel &a, cudaStream_t s);
template <class R>
cudaError_t launch_adjoint_gather(const DeviceModel &m, const AdjointModel &a, cudaStream_t s);
// gsum += gacc, gacc = 0 (mixed mode, at the end of each reversed segment).
template <class R>
cudaError_t launch_adjoint_fold(const DeviceModel &m, const AdjointModel &a, cudaStream_t s);
// After a forward step (node forces f_n in pdyn, step counter n): jacc[p] += sum_d seed_pd R_pd(t_n) / K
// with seed / K = -c, i.e. the particle's share of the objective.
cudaError_t launch_objective(const DeviceModel &m, const AdjointModel &a, cudaStream_t s);
// Device evaluation of the facet law and its vector-Jacobian product on independent inputs:
// in [n][16] = l, e(3), de(3), eV, t_old(3), e_max_old, E0, alpha, sigma_t, 0; adj_out [n][4];
// out [n][4] = t_new(3), e_max_new; adj_in [n][16] (same layout as in, slot 0 = 0).
template <class R>
cudaError_t launch_law_vjp(const LawConst<R> *law, int64_t n, const double *in, const double *adj_out, double *out,
                           double *adj_in, cudaStream_t s);
template <class R>
cudaError_t launch_hist_from_user(const DeviceModel &m, const double *in5, cudaStream_t s);

}  // namespace ldpm
