// Solve-phase kernels of the V-cycle (Alg. 2) shared by the single- and
// multi-right-hand-side paths.
#pragma once
#include "gmg_internal.cuh"

namespace gmg {

// Galerkin values, solve layout and coarsest inverse for the current level-0
// values.  With `defer` the inverse runs on the handle's own stream and the
// call returns once the Galerkin values are checked; later calls join it.
gmg_status numeric_setup(gmg_ctx* c, cudaStream_t s, bool defer = false);
gmg_status setup_impl(gmg_ctx* c, const gmg_csr* A, int nP, const gmg_prolong* P, const int32_t* const* coloring,
                      cudaStream_t s);

// level-vector selection by precision
template <class T> struct Vec;
template <> struct Vec<double> {
  static double* x(Level& L) { return L.x64; }
  static double* b(Level& L) { return L.b64; }
  static double* r(Level& L) { return L.r64; }
  static const double* v(const Ell& E) { return E.v64; }
  static const double* dinv(const Level& L) { return L.dinv64; }
  static const double* diag(const Level& L) { return L.diag64; }
  static const double* pw(const Level& L) { return L.p_w64; }
};
template <> struct Vec<float> {
  static float* x(Level& L) { return L.x32; }
  static float* b(Level& L) { return L.b32; }
  static float* r(Level& L) { return L.r32; }
  static const float* v(const Ell& E) { return E.v32; }
  static const float* dinv(const Level& L) { return L.dinv32; }
  static const float* diag(const Level& L) { return L.diag32; }
  static const float* pw(const Level& L) { return L.p_w32; }
};

// host launchers (gmg_cycle.cu)
template <class T> gmg_status launch_gs_colour(Level& L, int colour, const T* b, T* x, cudaStream_t s);
template <class T> gmg_status launch_residual(Level& L, const T* x, const T* b, T* r, cudaStream_t s);
// With dinvc, the rows of colour 0 of the coarse level (the first nc0) get
// x = b / a_ii (their first Gauss-Seidel update from zero) instead of 0.
template <class T> gmg_status launch_restrict(Level& L, const T* r, T* bc, T* xc, cudaStream_t s,
                                              const T* dinvc = nullptr, int64_t nc0 = 0);
template <class T> gmg_status launch_prolong(Level& L, const T* u, T* x, cudaStream_t s);
template <class T> gmg_status launch_coarse(gmg_ctx* c, const T* b, T* x, cudaStream_t s);
// MGI(x_l, b_l, l) on the level's own vectors, or on x_in / b_in (finest
// level only) when given.
template <class T> gmg_status vcycle(gmg_ctx* c, int l, cudaStream_t s, bool c0_done = false, T* x_in = nullptr,
                                     const T* b_in = nullptr);

gmg_status launch_d2f(int64_t n, const double* a, float* b, cudaStream_t s);
gmg_status launch_f2d(int64_t n, const float* a, double* b, cudaStream_t s);
// check: run the convergence test of the device-side loop (condition h) at
// the end of the iteration where the iteration's kernels allow it.
gmg_status iteration_body(gmg_ctx* c, int mode, int seg, cudaStream_t s, cudaGraphConditionalHandle h = 0,
                          bool check = false);
gmg_status pcg_start(gmg_ctx* c, int mode, cudaStream_t s);
gmg_status outer_residual_norm(gmg_ctx* c, cudaStream_t s);
gmg_status norm_b(gmg_ctx* c, cudaStream_t s);
enum { S_NB2 = 0, S_RR = 1, S_RZ = 2, S_PQ = 3, S_NUM = 4, S_RZN = 5, S_BETA = 6, S_TOL = 7 };
// One iteration of the device-side loop (PCG: segment 1 of the previous
// iteration, then segment 0) followed by the convergence test that sets the
// loop's condition `h` (captured into the body of a WHILE node).
gmg_status loop_body(gmg_ctx* c, int mode, cudaGraphConditionalHandle h, cudaStream_t s);
gmg_status launch_gather(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t s);
gmg_status launch_scatter(int64_t n, const int32_t* perm, const double* src, double* dst, cudaStream_t s);

}  // namespace gmg
