// Internal records shared by the kernel and host translation units of the
// GB300 explicit PDN impact step.  Not part of the public C ABI (pdn.h).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pdn {

// Contact-surface nodes per block of the contact kernel, and per run of the
// active-node counts it writes (Dev::act_cnt): 16 flag words of 16 nodes.
constexpr int kActRun = 256;

// Device-side state machine of a pass.  A pass is one launch of the five step
// kernels (contact, hex, interface, gather, tail); the tail decides whether
// the next pass advances to a new step or repeats the current one after
// releasing adhesive contact nodes (Algorithm 2).
enum Mode : int32_t {
  MODE_ADVANCE = 0,  // next pass computes a new step
  MODE_REPEAT = 1,   // next pass repeats the current step with released nodes
  MODE_PRIME = 2,    // next pass recomputes the acceleration of an installed state
  MODE_FORCES = 3,   // next pass evaluates internal forces of the committed state
  MODE_DONE = 4,     // target step reached: passes are no-ops
  MODE_HALT = 5      // sticky error: passes are no-ops
};

struct Ctl {
  int32_t mode;
  int32_t dpar;        // node buffer holding the current pass's displacement
  int32_t hpar;        // history buffer holding the committed history
  int32_t repeats;     // repetitions of the current step so far
  int32_t status;      // 0 or a PDN_E_* code
  int32_t max_repeats;
  int64_t step;        // committed steps
  int64_t target;      // step at which passes stop
  int64_t n_active;    // contact nodes of the last committed step
  int64_t n_repeats_total;
  int64_t hist_count;  // contact-force samples written
  double time;
  double f_peak;
  int32_t nonfinite;   // set by the gather when an acceleration is not finite
  int32_t timeout;     // set by a kernel whose bounded wait on the tensor core gave up
  int32_t check;       // first failed device bounds check of a PDN_CHECK build (CheckCode), else 0
  int32_t pad;
};

// Device bounds checks of a library built with PDN_CHECK defined: an index
// out of range records its code in Ctl::check, the item skips the access, and
// the tail halts the run (PDN_E_ARG).  Without PDN_CHECK the checks compile
// to nothing.
enum CheckCode : int32_t {
  CHECK_ELEMENT_NODE = 1,  // a hex or interface element names a node outside [0, n_nodes)
  CHECK_SURFACE_NODE = 2   // a contact-surface entry names a node outside [0, n_nodes)
};

// Rigid striker (Sec. 2.2.2).  The committed part is written only by the tail
// kernel; every pass recomputes the step-(n+1) state from it.
struct Striker {
  double c[3], w[3];  // centre and velocity at the committed step n
  double F[3];        // contact force on the plate at step n: sum_j lambda_j n_j
  double axis[3];     // unit impact direction (the only free degree of freedom)
  double R, M;
  double iM;  // 1 / M, set with M (the per-pass update then needs no FP64 division)
  double g[3];
  int32_t has;
  int32_t pad;
};

// Striker state of the step being computed (n+1) and the acceleration used
// over it; written by the contact kernel, read by gather and tail.
struct StrikerStep {
  double c[3], w[3], aI[3];
};

constexpr int kMaxPlies = 64;

// Material constants in the element precision T (computed once on the host).
template <typename T>
struct Mat {
  // undamaged stiffness (ply axes, Voigt 11 22 33 12 13 23)
  T C11, C12, C13, C22, C23, C33, G12, G13, G23;
  // undamaged compliance, normal block
  T h11, h22, h33, h12, h13, h23;
  T E1, E2;
  T XT, XC, YT, YC, SL;
  T GXT, GXC, GYT, GYC, GSL;
  T ca, sa, etaT, ST, etaLc;  // fracture-plane constants; etaL = SL * etaLc
  T g;                        // GYT / GSL
  T Sp, Kp;
  // derived: 1 - g, 1/XC, 1/ST^2, ca (sa - etaT ca), Kp G12, 1/(G12 (1 + Kp))
  T g1, iXC, iST2, kT, KpG12, iG1Kp;
  // interface
  T KI, Ksh, KI_D3o2, Ksh_Dsho2, KI_D3oD3c, Ksh_DshoDshc, eta, onset_floor;
  T spread;
  T ply_c[kMaxPlies], ply_s[kMaxPlies];
  uint64_t seed;
  int32_t damage_on, plasticity_on;
};

// Column sweep of a layered plate (every hex and interface layer a full
// nx x ny grid of columns, nodes numbered layer by layer, x fastest): one
// launch evaluates the elements of a tile of columns layer by layer, bottom to
// top, sums the forces of the nodes whose elements all lie in the tile in
// shared memory (in the same order as the gather) and updates those nodes at
// once; only the nodes on tile boundaries (and on the boundaries of the
// z-chunks the sweep is split into) go through the element-force slots and a
// gather over their list.
constexpr int kMaxStages = 128;
struct Sweep {
  int32_t nx, ny;          // element columns
  int32_t nxn;             // node columns along x (nx + 1)
  int32_t n_stages;        // element layers, bottom to top
  int64_t per_layer;       // nodes per node layer
  int32_t tile;            // tile shape: 0 = 16 x 8, 1 = 8 x 8, 2 = 8 x 4 columns
  int32_t tiles_x, tiles_y;
  int32_t chunk_len;       // stages per z-chunk (the last may be shorter)
  int32_t chunks;
  int32_t pad;
  const int32_t *bnodes;   // nodes updated by the gather over the list (ascending)
  int64_t n_bnodes;
  int32_t kind[kMaxStages];  // 0 hex layer, 1 interface layer
  int32_t base[kMaxStages];  // first element id of the layer (hex or interface numbering)
  int32_t bot[kMaxStages];   // bottom node layer; the top one is bot + 1
};

template <typename T>
struct Vec4T;
template <>
struct Vec4T<float> {
  using type = float4;
};
template <>
struct Vec4T<double> {
  using type = double4_32a;  // 32-byte aligned: one 256-bit access per node
};

constexpr int kMaxPairLayers = 128;  // node layers a layered numbering may have

// Pointers of a context's device state for the step kernels.
template <typename T>
struct Dev {
  using V4 = typename Vec4T<T>::type;
  int64_t nn, nh, nc, ns;
  // mesh
  const int32_t *hex;      // [nh][8]
  const int32_t *coh;      // [nc][8]
  const int8_t *ply;       // [nh]
  const V4 *X4;            // [nn] reference coordinates (x, y, z, 0) in T
  const uint8_t *nflag;    // [nn] bits 0-2 constraint, bit 3 contact surface
  const int32_t *surf;     // [ns]
  const int32_t *surf_of;  // [nn] surface index or -1
  const double *Xs;        // [3][ns] surface reference coordinates (FP64)
  const int32_t *row;      // [nn + 1] CSR of node -> element-force slot
  const int32_t *col;      // [nnz] slot = 8*e + k (hex), 8*(nh + c) + k (interface)
  const int32_t *pos;      // [nnz] inverse of col: CSR position of slot (e, k)
  // with eight slots per node (ell): per element (hexes, then interfaces)
  // the rank of each corner's slot in its node's eight, 3 bits per corner,
  // so that slot = 8 node + rank (null otherwise)
  const uint32_t *rank;
  const double *mass;      // [nn]
  const T *inv_mass;       // [nn]
  // state (double buffered)
  double *d[2], *v[2];     // [3][nn]
  V4 *u4[2];               // [nn] element-precision mirror of d
  T *hist[2];              // [7][8][nh] history per Gauss point
  T *rD[2];                // [4][nc] interface thresholds
  // 1 = every point of the element still holds the initial history (r = 1,
  // plastic strain 0; interface r_D = 0): its history is neither read nor
  // written.  Double-buffered with the history; nullptr = no flags (history
  // always read and written).
  uint8_t *pflag[2];       // [nh]
  uint8_t *cflag[2];       // [nc]
  V4 *fe;                  // [(nh + nc) * 8] element nodal forces
  // contact
  uint8_t *act[2];         // [ns] contact set by step parity
  uint8_t *rel;            // [ns] released in the current step
  // active contact nodes of each run of kActRun consecutive surface nodes,
  // written by the contact kernel of every stepping pass and read by the
  // tail of the same pass (null: the tail counts the flag words itself)
  int32_t *act_cnt;        // [ceil(ns / kActRun)]
  // local repetition of a step: marks of the elements ([nh + nc], hexes then
  // interfaces) and nodes ([nn]) that a repeated pass evaluates again; zero
  // outside a repeated pass (null: repeated passes evaluate everything)
  uint8_t *rmark_e;
  uint8_t *rmark_n;
  double *nrm;             // [3][ns]
  double *lam;             // [ns]
  double *trial;           // [6][ns] pre-projection d and v of active nodes
  // control
  Ctl *ctl;
  Striker *imp;
  StrikerStep *imp_step;
  double *fhist;           // [hist_cap]
  int64_t hist_cap;
  double *fout;            // [3][nn] internal force output (MODE_FORCES)
  // integration
  double dt, phi;
  double grav[3];
  T grav_t[3];  // gravity in the element precision
  // every hex is an axis-aligned box whose corner coordinates coincide
  // exactly in pairs (in T): the trilinear map is affine and J is constant
  int32_t all_boxes;
  // every interface element's lower face is an axis-aligned rectangle in a
  // plane z = const, corners counter-clockwise from +z, coordinates equal in
  // pairs exactly (in T): the local frame is the global axes and every
  // point's area weight is a quarter of the rectangle
  int32_t all_flat_coh;
  // element-force slots: 1 = eight per node (slot 8 j + k holds the k-th
  // entry of node j's CSR row, the rest stay zero), 0 = CSR positions
  int32_t ell;
  // launch configuration picked by the autotuner: hex occupancy variant
  // (0: 4 blocks of 128 per SM, 1: 5, 2: 6, 3: 3).  The variants execute the
  // same source; results can differ at FP32 rounding between variants (the
  // assembler's multiply-add contraction depends on the register budget).
  int32_t hex_variant;
  // learned law (FP32 box elements only): the network's parameters followed
  // by its scaling (include/pdn_surrogate.h), or nullptr for the exact law;
  // points whose squared loading-function ratio exceeds sur_ratio2 (or whose
  // inputs leave the training box) take the exact law
  const float *sur_params;
  float sur_ratio2;
  // the first node id when the contact surface is the ascending contiguous
  // range surf[s] = surf_base + s (then s and j convert without the index
  // arrays), else -1
  int32_t surf_base;
  // column sweep of the pass (FP32 box hexes, flat interfaces, eight slots
  // per node), or nullptr for separate element and gather kernels; a host
  // pointer, read only by the launcher
  const Sweep *sweep;
  // Interfaces as node pairs.  With Newton-Cotes points at the corners and
  // the global frame of flat interfaces, the traction at a point of an
  // interface element depends only on the displacement jump of the two
  // coincident nodes there (and the point's threshold r_D), and every
  // element sharing that node pair sees the same jump and the same history.
  // The gather then evaluates the cohesive law once per node and adds each
  // incident element's share w tau in CSR order, with no interface kernel
  // and no interface slots.  Per node {partner node or -1, meta}: meta bits
  // 0-2 incident interface elements, bit 3 the node is on the upper face,
  // bits 4-7 incident hexes (their slots come first).  nullptr: interface
  // elements (k_coh).
  const int2 *ipair;
  // area weights of the incident interface elements in CSR order ([nn]),
  // or nullptr when every weight equals coh_w
  const V4 *iw;
  T coh_w;
  // threshold r_D of each node pair, stored at its lower node ([nn],
  // double-buffered with the history); the element layout rD/cflag is
  // written from it only for the readers (history, energy, damage field)
  T *rDn[2];
  // Node pairs of a layered numbering (every block of pair_layer consecutive
  // node ids is one node layer, and the partner of an interface node is the
  // same position in the layer above or below): the gather then knows a
  // node's partner from its id and loads everything in one round.  Bit l of
  // pair_mask[0] / pair_mask[1] (words of 64 layers): layer l is the lower /
  // upper side of an interface; node flag bits 4-6 hold the count of a node's
  // interface elements.  0: partners from ipair (a second load round).
  int32_t pair_layer;
  uint64_t pair_mask[2][2];
  // compact force slots of a layered numbering with node pairs: a node of an
  // interface layer owns 4 slots (it has at most four hexes and its
  // interface elements write none), any other node 8; layer l starts at slot
  // L (8 l - 4 (interface layers below l)).  0: 8 slots per node
  int32_t slot_compact;
  // with compact slots: the first slot of node j of layer l is
  // j * width(l) + layer_off[l] (width 4 on interface layers, 8 else), and
  // l = j / pair_layer, found as the rounded product with pair_inv_L
  // corrected by one either way
  float pair_inv_L;
  int32_t layer_off[kMaxPairLayers];
};
constexpr int kFlagPairShift = 4;  // node flag bits 4-6: incident interface elements

// Launchers (pdn_kernels.cu).
template <typename T>
cudaError_t launch_pass(const Dev<T> &D, const Mat<T> &M, cudaStream_t s, int32_t gather_block,
                        cudaEvent_t *ev /* [6] or nullptr */, cudaStream_t side = nullptr,
                        cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
cudaError_t launch_striker_init(Striker *S, StrikerStep *ss, double dt, cudaStream_t s);
// Hex kernel with the learned law (pdn_surrogate.cu); D.sur_params != nullptr.
cudaError_t launch_hex_sur(const Dev<float> &D, const Mat<float> &M, cudaStream_t s);
template <typename T>
cudaError_t launch_damage_field(const Dev<T> &D, const Mat<T> &M, int which, float *out,
                                cudaStream_t s);
// Interfaces as node pairs: writes the element layout of the committed
// interface thresholds (rD, cflag) from the pairs' (no-op otherwise).
template <typename T>
cudaError_t launch_pairs_to_elements(const Dev<T> &D, cudaStream_t s);

}  // namespace pdn
