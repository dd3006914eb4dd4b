// Spectral products of the system operator of Eq. (sys) at one frequency
// node: from the seven source spectra (J_x, J_y, J_z, M_x, M_y, M_z, rho) and
// the kernel spectra (G, dG/dx, dG/dy, dG/dz) to the four result spectra
//   A_a = j k0 G J_a - (grad G x M)_a   (a = x, y, z),   Phi = G rho,
// the grid form of the L_A and K terms of Eq. (AIM_Lin) and of the charge
// potential.  C = double2 (FP64) or float2 (complex64 grid path), R its real type.
#pragma once
#include <cuda_runtime.h>

namespace sie {

template <class C>
__device__ __forceinline__ C sm_mul(C a, C b)
{
    C t;
    t.x = a.x * b.x - a.y * b.y;
    t.y = a.x * b.y + a.y * b.x;
    return t;
}

template <class C, class R>
__device__ __forceinline__ void sys_specmul(C G, C gx, C gy, C gz, R k0, const C* in, C* out)
{
    C jG;
    jG.x = -k0 * G.y;  // j k0 G
    jG.y = k0 * G.x;
    const C mx = in[3], my = in[4], mz = in[5];
    const C cx = sm_mul(gy, mz), cy = sm_mul(gz, mx), cz = sm_mul(gx, my);
    const C dx = sm_mul(gz, my), dy = sm_mul(gx, mz), dz = sm_mul(gy, mx);
    const C a0 = sm_mul(jG, in[0]), a1 = sm_mul(jG, in[1]), a2 = sm_mul(jG, in[2]);
    out[0].x = a0.x - (cx.x - dx.x);
    out[0].y = a0.y - (cx.y - dx.y);
    out[1].x = a1.x - (cy.x - dy.x);
    out[1].y = a1.y - (cy.y - dy.y);
    out[2].x = a2.x - (cz.x - dz.x);
    out[2].y = a2.y - (cz.y - dz.y);
    out[3] = sm_mul(G, in[6]);
}

}  // namespace sie
