// lb_internal.h -- context object and the host-side launcher interface between
// the C ABI (lb_capi.cu) and the kernel translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/lb.h"

namespace lbgb {

// Kernel-facing description of one domain in internal coordinates (see
// lb_lattice.cuh: 2D grids are nx x 1 x ny internally).
struct Geometry {
  int lattice, q, d;
  int nx, ny, nz;          // internal extents
  int64_t pitch;           // elements per stored row (>= nx, multiple of 32)
  int64_t vol;             // elements per population: pitch * ny * nz
  int per[3];              // periodic flag per internal axis
  int zlink[2];            // internal -z / +z face borders another slab (LB_LINK)
  int face_kind[6];        // internal faces -x,+x,-y,+y,-z,+z
  double wall_u[6][3];     // internal components
  double tau, rho0;
  double force[3];         // internal components
  bool has_force;
};

// Brick decomposition and shell layout of the fused scheme.
struct FusedPlan {
  int bx, by, bz;          // brick cross-section and sweep length
  int nbx, nby, nbz;
  int nxf, nyf, nzf;       // directions crossing an x / y / z face (per side)
  int zg;                  // 1: ghost planes / brick rows for link faces (see K1Args)
  int64_t sx_elems, sy_elems, sz_elems;  // per parity
  int64_t parity_elems;
  int slots;               // TMA pipeline depth
  int wbuf;                // shared window buffers (2: one barrier per plane)
  int xwarps;              // dedicated export warps (0: node-owning warps export)
  int npt;                 // nodes per thread (1 scalar, 2 paired FP32x2 kernel)
  int ts;                  // 1: completed planes leave through a TMA store
  int minb;                // CTAs per SM the compiled shape is built for
  size_t smem_bytes;
};

struct Status;

}  // namespace lbgb

struct lb_ctx {
  lbgb::Geometry g;
  lb_boundary bnd_user;   // the creation arguments as given (for proxies of the autotuner)
  lb_options opt_user;
  double tau_user;
  int32_t lattice, storage, scheme;
  int64_t dims[3];
  int64_t n_nodes;
  int device;
  cudaStream_t stream;
  bool own_stream;
  size_t elem_bytes;      // storage element size
  size_t real_bytes;      // arithmetic element size (shells, moments)
  void* f;                // the population array: q * vol elements
  size_t f_bytes;
  void* aux;              // shells (fused) or moment arrays (two-pass)
  size_t aux_bytes;
  lbgb::FusedPlan plan;
  int parity;             // shell parity holding the current post-collision halo
  CUtensorMap tmap;       // TMA descriptor of the population array (fused)
  int* d_status;          // sticky device status word
  double* d_red;          // reduction partials
  float* d_uprev;         // residual snapshot, allocated on first use
  bool have_uprev;
  int64_t steps_done;
  // two fused steps captured as a CUDA graph from shell parity graph_parity
  // (lb_step replays it for long runs; null until first needed, dropped when
  // the brick plan or the shell buffers change)
  cudaGraphExec_t step_graph = nullptr;
  int graph_parity = 0;
};

namespace lbgb {

// ---- two-pass scheme (lb_k0.cu)
cudaError_t k0_step(lb_ctx* ctx);
size_t k0_aux_bytes(const Geometry& g, int storage);
cudaError_t k0_step_buffers(const Geometry& g, double* ft, double* mom, cudaStream_t stream);

// ---- fused scheme (lb_k1_*.cu)
// sms > 0 plans for that many SMs instead of the current device's count
bool k1_plan(const Geometry& g, int storage, const int32_t tile_req[3], FusedPlan* plan, int sms = 0);
// plan with one given compiled shape (a K1Variant*, see lb_k1_launch.cuh) and
// sweep length bz (0 = the planner's choice)
bool k1_plan_variant(const Geometry& g, const void* variant, int bz, FusedPlan* plan);
// compiled shapes for (lattice, storage), in the planner's order; returns the count
int k1_variants_for(int lattice, int storage, const void** out, int cap);
// switch a fused-scheme context to another compiled shape and sweep length
// (bz = 0: the planner's choice): new shell buffers and TMA descriptor, shell
// rebuilt from the current populations (lb_capi.cu)
int ctx_replan(lb_ctx* ctx, const void* variant, int bz = 0);
// release the captured step pair of lb_step (plan or shell buffers change)
void drop_step_graph(lb_ctx* ctx);
cudaError_t k1_step(lb_ctx* ctx);
cudaError_t k1_bootstrap(lb_ctx* ctx);  // fill the current shell parity from f
cudaError_t k1_configure(lb_ctx* ctx);  // one-time kernel attributes

// ---- state conversion, readout and reductions (lb_aux.cu)
cudaError_t aux_set_populations(lb_ctx* ctx, const double* f_dev);
cudaError_t aux_get_populations(lb_ctx* ctx, double* f_dev);
cudaError_t aux_init_moments(lb_ctx* ctx, const double* rho, const double* u, const double* pineq);
cudaError_t aux_init_uniform(lb_ctx* ctx, double rho, const double u_user[3]);
cudaError_t aux_moments(lb_ctx* ctx, double* rho, double* u);
// the same for nodes [n0, n1) only, with buffers holding element idx - n0 of
// each component and components cs elements apart
cudaError_t aux_init_moments_range(lb_ctx* ctx, const double* rho, const double* u, const double* pineq, int64_t n0,
                                   int64_t n1, int64_t cs);
cudaError_t aux_moments_range(lb_ctx* ctx, double* rho, double* u, int64_t n0, int64_t n1, int64_t cs);
cudaError_t aux_get_region(lb_ctx* ctx, const int64_t lo[3], const int64_t size[3], double* f_dev);
cudaError_t aux_reduce(lb_ctx* ctx, double* host_out /* mass, mom[3], du2, u2, nonfinite */,
                       bool residual);
// the same sums enqueued on `stream`, the seven values written to dev_out
// (device memory); nothing is copied to the host or synchronised
cudaError_t aux_reduce_enqueue(lb_ctx* ctx, cudaStream_t stream, double* dev_out, bool residual);
constexpr int kReduceFields = 7;
// lb_reduce's outputs from the seven sums of aux_reduce (lb_capi.cu); returns
// LB_E_DIVERGED if a value is not finite
int reduce_finish(lb_ctx* ctx, const double* sums, bool want_residual, double* mass, double mom[3],
                  double* residual);

// map a user-facing (canonical) vector to internal axes and back
void to_internal(int d, const double in[3], double out[3]);
int internal_axis_of_user(int d, int user_axis);

}  // namespace lbgb
