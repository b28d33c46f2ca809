// Real spherical-harmonic basis to degree 3 (Condon-Shortley signs, as the
// 3DG-S renderer), for device and host, in float or double.
#pragma once

#define SH_C0 0.28209479177387814
#define SH_C1 0.4886025119029199
#define SH_C2A 1.0925484305920792
#define SH_C2B 0.31539156525252005
#define SH_C2C 0.5462742152960396
#define SH_C3A 0.5900435899266435
#define SH_C3B 2.890611442640554
#define SH_C3C 0.4570457994644658
#define SH_C3D 0.3731763325901154
#define SH_C3E 1.445305721320277

namespace gs3 {

// Y[(deg + 1)^2] at the unit direction (x, y, z)
template <typename T>
__host__ __device__ __forceinline__ void sh_basis_t(int deg, T x, T y, T z, T *Y)
{
    Y[0] = T(SH_C0);
    if (deg < 1) return;
    Y[1] = -T(SH_C1) * y;
    Y[2] = T(SH_C1) * z;
    Y[3] = -T(SH_C1) * x;
    if (deg < 2) return;
    T xx = x * x, yy = y * y, zz = z * z;
    Y[4] = T(SH_C2A) * x * y;
    Y[5] = -T(SH_C2A) * y * z;
    Y[6] = T(SH_C2B) * (T(2) * zz - xx - yy);
    Y[7] = -T(SH_C2A) * x * z;
    Y[8] = T(SH_C2C) * (xx - yy);
    if (deg < 3) return;
    Y[9] = -T(SH_C3A) * y * (T(3) * xx - yy);
    Y[10] = T(SH_C3B) * x * y * z;
    Y[11] = -T(SH_C3C) * y * (T(4) * zz - xx - yy);
    Y[12] = T(SH_C3D) * z * (T(2) * zz - T(3) * xx - T(3) * yy);
    Y[13] = -T(SH_C3C) * x * (T(4) * zz - xx - yy);
    Y[14] = T(SH_C3E) * z * (xx - yy);
    Y[15] = -T(SH_C3A) * x * (xx - T(3) * yy);
}

}  // namespace gs3
