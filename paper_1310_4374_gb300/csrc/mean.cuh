// Newtonian potential of a uniform box, for the mean of phi_near (App. C).
#pragma once

namespace psum {

// ---------------------------------------------------------------------------
// Mean of phi_near over the box (Eq. pfx4).  The near block is the union of the
// box images, so sum_p Phi_0(x + p) = U(x) / V0 with U(x) = int_B dV(y)/|y - x|
// over the block B = [-H0,H0] x [-H1,H1] x [-H2,H2].  U is reduced to the faces
// by the divergence theorem (Eqs. B1-B2), each face integral to its four edges
// by the divergence theorem in the plane (Eqs. B3-B5), and each edge integral
// has the primitive (Eqs. B7-B9, in the form derived below)
//   G(t; z, h) = z ln(t + rho) + h atan(h t / (z rho)) - h atan(t / z),
//   rho = sqrt(t^2 + z^2 + h^2),
// where h is the distance from x to the face plane, z the signed distance of
// the projected point to the edge line (positive inside the face) and t runs
// along the edge from the foot of the perpendicular.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ double edge_primitive(double t, double z, double h) {
    const double rho = sqrt(t * t + z * z + h * h);
    const double lg = t >= 0.0 ? log(t + rho) : log((z * z + h * h) / (rho - t));
    return z * lg + h * atan(h * t / (z * rho)) - h * atan(t / z);
}

__host__ __device__ __forceinline__ double edge_integral(double z, double h, double t0, double t1) {
    if (z == 0.0) return 0.0;     // the point projects onto the edge line: the integrand vanishes
    return edge_primitive(t1, z, h) - edge_primitive(t0, z, h);
}

__host__ __device__ __forceinline__ double block_potential(const double X[3], const double H[3]) {
    double U = 0.0;
    for (int k = 0; k < 3; ++k) {
        const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const double a = X[k1], b = X[k2];
        // face integral L = sum over its four edges (independent of the face's side)
        const double h_lo = fabs(H[k] + X[k]), h_hi = fabs(H[k] - X[k]);
        for (int side = 0; side < 2; ++side) {
            const double s = side ? (H[k] - X[k]) : (H[k] + X[k]);     // n . (y - x) on the face
            const double h = side ? h_hi : h_lo;
            if (s == 0.0) continue;
            double L = 0.0;
            L += edge_integral(H[k1] - a, h, -H[k2] - b, H[k2] - b);
            L += edge_integral(H[k1] + a, h, -H[k2] - b, H[k2] - b);
            L += edge_integral(H[k2] - b, h, -H[k1] - a, H[k1] - a);
            L += edge_integral(H[k2] + b, h, -H[k1] - a, H[k1] - a);
            U += 0.5 * s * L;
        }
    }
    return U;
}


}  // namespace psum
