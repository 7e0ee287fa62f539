// Coefficient-map access policies of the 2D step kernels.
//
// DenseMaps<T>: one value per cell for every map (float or bf16 storage).
// IdxMaps: one uint8 tissue index per cell; every cell coefficient comes from
//   per-tissue float tables (256 entries at most) staged in shared memory,
//   the reduced-storage form of the medium.  C-PML strips stay per cell.
// Both expose the same operations on a 4-cell group (a Cell).
#pragma once
#include "fw2_internal.cuh"

namespace fw2 {

// Table layout of the index form: [field][kTissues] floats, fields in this
// order (then a1[nu], b1[nu], a2[nu], b2[nu] for nu < N).
enum { kTabK = 0, kTabRho = 1, kTabChi = 2, kTabIk1 = 3, kTabIk2 = 4, kTabRelax = 5 };
constexpr int kTissues = 256;
constexpr int kTableFields = kTabRelax + 4 * kTabSlots;

template <typename T>
struct DenseMaps {
  using StripT = T;
  static constexpr int kSmemFloats = 1;
  struct Cell {
    long long c;
  };
  const T *K, *rho, *chi, *ik1_, *ik2_, *a1_, *b1_, *a2_, *b2_;
  long long S;
  const float *ms;  // map scales (FP16 storage; ignored by float and bf16 loads)
  __device__ __forceinline__ explicit DenseMaps(const StepParams &P)
      : K(static_cast<const T *>(P.K)), rho(static_cast<const T *>(P.rho)), chi(static_cast<const T *>(P.chi)),
        ik1_(static_cast<const T *>(P.ik1)), ik2_(static_cast<const T *>(P.ik2)),
        a1_(static_cast<const T *>(P.a1)), b1_(static_cast<const T *>(P.b1)),
        a2_(static_cast<const T *>(P.a2)), b2_(static_cast<const T *>(P.b2)), S(P.npts_alloc), ms(P.ms) {}
  __device__ __forceinline__ void stage(const StepParams &, float *, int) const {}
  __device__ __forceinline__ void bind(const float *) {}
  __device__ __forceinline__ Cell cell(long long c) const { return {c}; }
  __device__ __forceinline__ float rho_at(long long gidx) const { return ldmap(rho, gidx, ms[kMsRho]); }
  __device__ __forceinline__ float K_at(long long gidx) const { return ldmap(K, gidx, ms[kMsK]); }
  __device__ __forceinline__ float4 Kv(Cell x) const { return ldmap4(K, x.c, ms[kMsK]); }
  __device__ __forceinline__ float4 chiv(Cell x) const { return ldmap4(chi, x.c, ms[kMsChi]); }
  __device__ __forceinline__ float4 ik1(Cell x) const { return ldmap4(ik1_, x.c, ms[kMsIk1]); }
  __device__ __forceinline__ float4 ik2(Cell x) const { return ldmap4(ik2_, x.c, ms[kMsIk2]); }
  template <int OP>
  __device__ __forceinline__ float4 a(Cell x, int nu) const {
    return ldmap4(OP == 1 ? a1_ : a2_, nu * S + x.c, ms[(OP == 1 ? kMsA1 : kMsA2) + nu]);
  }
  template <int OP>
  __device__ __forceinline__ float4 b(Cell x, int nu) const {
    return ldb4(OP == 1 ? b1_ : b2_, nu * S + x.c, ms[(OP == 1 ? kMsB1 : kMsB2) + nu]);
  }
  // single cell e of the group (edge paths)
  template <int OP>
  __device__ __forceinline__ float a1c(Cell x, int nu, int e) const {
    return ldmap(OP == 1 ? a1_ : a2_, nu * S + x.c + e, ms[(OP == 1 ? kMsA1 : kMsA2) + nu]);
  }
  template <int OP>
  __device__ __forceinline__ float b1c(Cell x, int nu, int e) const {
    return ldb(OP == 1 ? b1_ : b2_, nu * S + x.c + e, ms[(OP == 1 ? kMsB1 : kMsB2) + nu]);
  }
};

struct IdxMaps {
  using StripT = float;
  static constexpr int kSmemFloats = kTissues * kTableFields;
  struct Cell {
    uchar4 t;
  };
  const unsigned char *idx;
  const float *tab;  // table in shared memory once bound
  __device__ __forceinline__ explicit IdxMaps(const StepParams &P) : idx(P.tissue), tab(nullptr) {}
  // copy the per-tissue table (global, [field][256]) into shared memory
  __device__ __forceinline__ void stage(const StepParams &P, float *s, int tid) const {
    const float4 *src = reinterpret_cast<const float4 *>(P.table);
    float4 *dst = reinterpret_cast<float4 *>(s);
    constexpr int n4 = kTableFields * kTissues / 4;
    for (int t = tid; t < n4; t += 256) dst[t] = __ldg(src + t);
  }
  __device__ __forceinline__ void bind(const float *s) { tab = s; }
  __device__ __forceinline__ Cell cell(long long c) const {
    return {__ldg(reinterpret_cast<const uchar4 *>(idx + c))};
  }
  __device__ __forceinline__ float4 look(int field, Cell x) const {
    const float *f = tab + field * kTissues;
    return make_float4(f[x.t.x], f[x.t.y], f[x.t.z], f[x.t.w]);
  }
  __device__ __forceinline__ float rho_at(long long gidx) const {
    return tab[kTabRho * kTissues + __ldg(idx + gidx)];
  }
  __device__ __forceinline__ float K_at(long long gidx) const { return tab[kTabK * kTissues + __ldg(idx + gidx)]; }
  __device__ __forceinline__ float4 Kv(Cell x) const { return look(kTabK, x); }
  __device__ __forceinline__ float4 chiv(Cell x) const { return look(kTabChi, x); }
  __device__ __forceinline__ float4 ik1(Cell x) const { return look(kTabIk1, x); }
  __device__ __forceinline__ float4 ik2(Cell x) const { return look(kTabIk2, x); }
  // relaxation fields: a1[nu] at kTabRelax + nu, b1 at + N, a2 at + 2N, b2 at + 3N
  // (kTabSlots slots reserved; the prep fills the first n_relax of each)
  template <int OP>
  __device__ __forceinline__ float4 a(Cell x, int nu) const {
    return look(kTabRelax + (OP == 1 ? 0 : 2 * kTabSlots) + nu, x);
  }
  template <int OP>
  __device__ __forceinline__ float4 b(Cell x, int nu) const {
    return look(kTabRelax + (OP == 1 ? kTabSlots : 3 * kTabSlots) + nu, x);
  }
  template <int OP>
  __device__ __forceinline__ float a1c(Cell x, int nu, int e) const {
    return el(a<OP>(x, nu), e);
  }
  template <int OP>
  __device__ __forceinline__ float b1c(Cell x, int nu, int e) const {
    return el(b<OP>(x, nu), e);
  }
};

// IdxMaps16: one uint16 tissue index per cell (up to 65536 tissues); the
// per-tissue tables ([field][tab_stride] floats, up to 5.5 MB) stay in global
// memory and are read through L2 and the read-only cache.  Same table values
// and arithmetic as IdxMaps.
struct IdxMaps16 {
  using StripT = float;
  static constexpr int kSmemFloats = 1;
  struct Cell {
    ushort4 t;
  };
  const unsigned short *idx;
  const float *tab;
  int S;  // field stride of the table
  __device__ __forceinline__ explicit IdxMaps16(const StepParams &P)
      : idx(reinterpret_cast<const unsigned short *>(P.tissue)), tab(P.table), S(P.tab_stride) {}
  __device__ __forceinline__ void stage(const StepParams &, float *, int) const {}
  __device__ __forceinline__ void bind(const float *) {}
  __device__ __forceinline__ Cell cell(long long c) const {
    return {__ldg(reinterpret_cast<const ushort4 *>(idx + c))};
  }
  __device__ __forceinline__ float at(int field, int t) const { return __ldg(tab + field * S + t); }
  __device__ __forceinline__ float4 look(int field, Cell x) const {
    return make_float4(at(field, x.t.x), at(field, x.t.y), at(field, x.t.z), at(field, x.t.w));
  }
  __device__ __forceinline__ float rho_at(long long gidx) const { return at(kTabRho, __ldg(idx + gidx)); }
  __device__ __forceinline__ float K_at(long long gidx) const { return at(kTabK, __ldg(idx + gidx)); }
  __device__ __forceinline__ float4 Kv(Cell x) const { return look(kTabK, x); }
  __device__ __forceinline__ float4 chiv(Cell x) const { return look(kTabChi, x); }
  __device__ __forceinline__ float4 ik1(Cell x) const { return look(kTabIk1, x); }
  __device__ __forceinline__ float4 ik2(Cell x) const { return look(kTabIk2, x); }
  template <int OP>
  __device__ __forceinline__ float4 a(Cell x, int nu) const {
    return look(kTabRelax + (OP == 1 ? 0 : 2 * kTabSlots) + nu, x);
  }
  template <int OP>
  __device__ __forceinline__ float4 b(Cell x, int nu) const {
    return look(kTabRelax + (OP == 1 ? kTabSlots : 3 * kTabSlots) + nu, x);
  }
  template <int OP>
  __device__ __forceinline__ float a1c(Cell x, int nu, int e) const {
    return el(a<OP>(x, nu), e);
  }
  template <int OP>
  __device__ __forceinline__ float b1c(Cell x, int nu, int e) const {
    return el(b<OP>(x, nu), e);
  }
};

}  // namespace fw2
