// Device views of the structure's force data (springs in CSR rows per
// marker, tethers, bending lines) shared by the force and reverse-step kernels.
#pragma once
#include "ib_internal.cuh"

namespace ibgb {

template <class T> struct ForceArgs {
    int m;
    const T *d;                  // [3][m]
    const T *dlo;                // [3][m] low part of d (FP32 contexts: d + dlo), else null
    const int32_t *sp_off, *sp_j;
    const T *sp_k, *sp_L0, *sp_e0, *sp_c0;
    long long nnz;
    const T *tk;
    const int32_t *bslot, *bn;
    const T *bc;
    long long nb;
    const T *mf_dir;             // [3][m] external force direction or null
    const double *d_time;        // [t, body, marker amplitude at t, 0]
};

template <class T> inline ForceArgs<T> force_args(ib_ctx *c)
{
    auto &mk = c->mk;
    ForceArgs<T> a{};
    a.m = (int)mk.m;
    a.d = (const T *)mk.d;
    a.dlo = c->fp64 ? nullptr : (const T *)mk.d + 3 * mk.m;
    a.sp_off = mk.sp_off;
    a.sp_j = mk.sp_j;
    a.sp_k = (const T *)mk.sp_k;
    a.sp_L0 = (const T *)mk.sp_L0;
    a.sp_e0 = (const T *)mk.sp_e0;
    a.sp_c0 = (const T *)mk.sp_c0;
    a.nnz = mk.nnz;
    a.tk = (const T *)mk.tk;
    a.bslot = mk.bslot;
    a.bn = mk.bn;
    a.bc = (const T *)mk.bc;
    a.nb = mk.nb;
    a.mf_dir = (const T *)mk.mf_dir;
    a.d_time = c->d_time;
    return a;
}

}  // namespace ibgb
