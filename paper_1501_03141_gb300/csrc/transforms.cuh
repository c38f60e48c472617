// Plane-wave sphere <-> real-space grid transforms at Gamma (declarations).
//
// Two real fields a, b (two vectors of the real-coefficient layout) travel
// through one complex 3D FFT as C = a + i b.  The transform is pruned to the
// sphere: x-lines exist only for (n2, n3) columns that meet the sphere, y-lines
// only for the |n3| <= R3 planes, and the z-lines of a fixed-x slab carry the
// grid values.  Work is split in three launches:
//   column pass  : x-lines of every column, sphere <-> B1[item][i1][col]
//   slab pass    : for one (item, i1): y-lines and z-lines in shared memory,
//                  optionally with the local potential multiplied in between
//   column pass back : x-lines back to the sphere, Hermitian unpacking of the
//                  two real fields and a fused epilogue
#pragma once

#include "common.cuh"
#include "df64.cuh"

namespace pdep {

// One upper column (n2, n3) of the half space, with its mirror (-n2, -n3).
struct UCol {
  int n2, n3, R1, h0;  // x-extent [-R1, R1]; half index of the first member
  int col, mcol;       // indices in the full column list (mcol == col for (0,0))
};

// Device-side description of one system's sphere and grid.
template <typename R>
struct SphereDev {
  int N1, N2, N3, R3;
  int n_half, n_pw, n_col, n_ucol;
  const UCol* ucol;         // [n_ucol]
  const int2* slot;         // [2 R3 + 1]: (R2(n3), first full-column index)
  const double* g2;         // |G_k|^2, [n_half]
  const R* kin;             // |G_k|^2 / 2 in the kernel's precision, [n_half]
  const cpx<R>* tw1;        // exp(+2 pi i j/N1), j < N1
  const cpx<R>* tw2;
  const cpx<R>* tw3;
#ifdef PDEP_BOUNDS_CHECK
  unsigned* status = nullptr;  // device status word the bounds tests report to
#endif
};

// Bounds-checked builds: the sphere members and the columns of x-line c lie
// inside the tables (members h0 .. h0 + 2 R1 of a mirrored pair, h0 ..
// h0 + R1 - 1 of the self-mirrored (0, 0) line).  Always true otherwise.
template <typename R>
__device__ __forceinline__ bool ucol_in_range(const SphereDev<R>& s, const UCol& c) {
#ifdef PDEP_BOUNDS_CHECK
  const int members = c.col == c.mcol ? c.R1 : 2 * c.R1 + 1;
  bool ok = in_range(s.status, c.col, s.n_col) && in_range(s.status, c.mcol, s.n_col) &&
            in_range(s.status, c.R1, s.N1 / 2 + 1);
  if (members > 0)
    ok = ok && in_range(s.status, c.h0, s.n_half) && in_range(s.status, c.h0 + members - 1, s.n_half);
  return ok;
#else
  return true;
#endif
}

// Bounds-checked builds: the columns of y-line slot (R2, first) lie inside
// the column list.  Always true otherwise.
template <typename R>
__device__ __forceinline__ bool slot_in_range(const SphereDev<R>& s, int2 info) {
#ifdef PDEP_BOUNDS_CHECK
  return in_range(s.status, info.y, s.n_col) && in_range(s.status, info.y + 2 * info.x, s.n_col) &&
         in_range(s.status, info.x, s.N2 / 2 + 1);
#else
  return true;
#endif
}

// Which real vectors an FFT item packs: vectors are grouped; item w of a
// group takes members 2w and 2w+1 (the second may be absent).
struct ItemMap {
  int vecs_per_group;
  int items_per_group;
  const int* list = nullptr;  // optional explicit vector list (pairs of entries)
  int n_list = 0;             // listed vectors (the largest count when n_dev is set)
  const int* n_dev = nullptr; // device count of listed vectors (<= n_list): kernels read it
                              // at launch, so a launch sized for n_list can be enqueued or
                              // captured before the count is known
  __host__ __device__ int vec(int item, int slot) const { return vec(item, slot, n_list); }
  // with the listed-vector count nl (the device count when n_dev is set)
  __host__ __device__ int vec(int item, int slot, int nl) const {
    if (list) {
      int idx = 2 * item + slot;
      return idx < nl ? list[idx] : -1;
    }
    int g = item / items_per_group;
    int w = item - g * items_per_group;
    int idx = 2 * w + slot;
    return idx < vecs_per_group ? g * vecs_per_group + idx : -1;
  }
};

// The listed-vector count a kernel works with (read once per kernel; the
// map itself stays unmodified in parameter space).
__device__ __forceinline__ int listed_count(const ItemMap& m) {
  return (m.list && m.n_dev) ? *m.n_dev : m.n_list;
}
// Number of FFT items to process, given that count.
__device__ __forceinline__ int items_of(const ItemMap& m, int n_items, int nl) {
  return (m.list && m.n_dev) ? (nl + 1) / 2 : n_items;
}

// Per-component multiplier applied to sphere data on the way in / out.
enum CoefKind : int { COEF_ONE = 0, COEF_SQRT_COULOMB = 1 };

// Epilogue of the column pass back:
//   y = scale * coef(G) * (transform) + (kin * |G|^2/2 + shift[vec]) * x_in
//       (+ beta * y_old)
// R is the arithmetic type of the transform; vectors are stored in
// Io<R>::T (FP64 for the double-float transforms, else R itself).
template <typename R>
struct Epilogue {
  using T = typename Io<R>::T;
  T* y;                 // output vectors (real layout)
  long long ldy;
  const T* x_in;        // vectors for the diagonal term (may be null)
  long long ldx;
  const T* shift;       // per vector, indexed vec % shift_period (may be null)
  int shift_period;
  R scale;
  R kin;                // 0 or 1
  T beta;               // 0: overwrite
  int coef;             // CoefKind
};

// Grid source of the grid -> sphere slab pass: field = f(r) * (ga(r) + i gb(r))
template <typename R>
struct GridSrc {
  using T = typename Io<R>::T;
  const T* f;          // may be null (f = 1)
  long long f_stride;  // per group (item_map group)
  const T* g;          // ga/gb are vectors of g with stride g_stride
  long long g_stride;
};

enum SlabMode : int {
  SLAB_HPSI = 0,       // cols -> grid -> *V -> cols
  SLAB_TO_GRID = 1,    // cols -> grid, written as two real fields
  SLAB_FROM_GRID = 2,  // grid (GridSrc) -> cols
};

template <typename R>
struct SlabArgs {
  int mode;
  cpx<R>* b1;            // [n_items][N1][n_col]
  int n_items;
  const R* v;            // local potential [N_r] (HPSI), in the arithmetic type
  typename Io<R>::T* out;  // TO_GRID: two fields per item at vec(item,s)*out_stride
  long long out_stride;
  double out_scale;
  GridSrc<R> src;        // FROM_GRID (f: one grid per group, g: per-vector grids)
  ItemMap map;
  // HPSI: also accumulate dn_j(r) += dn_scale u_v(r) x_vj(r) for
  // every vector i = j * dn_nocc + v of the item (atomically; dn may be null)
  double* dn = nullptr;
  const double* u = nullptr;  // occupied grids [dn_nocc][dn_stride]
  int dn_nocc = 1;
  long long dn_stride = 0;
  double dn_scale = 0.0;
};

// Host launchers (stream-ordered; no synchronisation).  R = float, double or
// df (double-float arithmetic on FP64 vectors).
template <typename R>
cudaError_t launch_cols_fwd(const SphereDev<R>& s, const typename Io<R>::T* x, long long ldx,
                            ItemMap map, int n_items, int coef, cpx<R>* b1, cudaStream_t st);
template <typename R>
cudaError_t launch_slab(const SphereDev<R>& s, const SlabArgs<R>& a, cudaStream_t st);
template <typename R>
cudaError_t launch_cols_bwd(const SphereDev<R>& s, const cpx<R>* b1, ItemMap map, int n_items,
                            const Epilogue<R>& ep, cudaStream_t st);

// H x in FP32 by one fused launch (column scratch in shared memory) for the
// cubic grids 24^3 .. 48^3: the same result as cols_fwd + slab (HPSI) +
// cols_bwd with that epilogue.  hpsi_fused_smem returns its shared memory
// per block, 0 where the fused form does not apply.
// planes (0 = default) sets the x-planes transformed at once by a block (the
// autotuner's FFT batch; a power of two from 1 to 16 whose thread groups
// still cover a plane's y-lines, else the default is used).
size_t hpsi_fused_smem(const SphereDev<float>& s, int planes = 0);
int hpsi_fused_planes(const SphereDev<float>& s, int planes = 0);
cudaError_t launch_hpsi_fused(const SphereDev<float>& s, const float* x, long long ldx, ItemMap map,
                              int n_items, const float* v, const Epilogue<float>& ep,
                              cudaStream_t st, int planes = 0);

bool grid_supported(int N1, int N2, int N3);
cudaError_t upload_local_twiddles();
size_t slab_smem_bytes(int n_col, int R3, int N2, size_t elem);

}  // namespace pdep
