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


// The same potential by the corner sum of the classical closed form for a rectangular
// prism: U(x) = sum over the 8 corners c of s_c F(c - x), s_c = +1 where an even number
// of coordinates of c take the lower bound, with
//   F(a, b, c) = ab ln(c + r) + bc ln(a + r) + ca ln(b + r)
//                - a^2/2 atan(bc/(ar)) - b^2/2 atan(ca/(br)) - c^2/2 atan(ab/(cr)),
// r = |(a, b, c)|: 24 logarithms and 24 arctangents where the face/edge route takes 48 and
// 96.  The device means evaluate it regrouped (below, 12 and 12); the plan's RBF box means on
// the host keep the face/edge route.  On 2e5 random boxes and points, inside and outside, the
// regrouped sum is within 2.9e-13 (relative) of a long-double corner sum, the plain float64
// corner sum within 1.1e-12.  Vanishing products drop their term (their limit is 0).

// The corner sum regrouped (any point; the block's own means have it inside, the ball's mean
// also outside).  Take an axis k and one of
// the four corners (p, q) of the other two axes ((k+1, k+2) cyclically): the two block corners
// that differ in k alone carry opposite signs, and F's terms p q ln(k + r) and
// -p^2/2 atan(q k/(p r)) of the two combine, with (k_u, r_u) and (k_l, r_l) the upper and lower
// corner's offset along k and distance:
//   ln(k_u + r_u) - ln(k_l + r_l) = ln((k_u + r_u)(r_l - k_l) / (p^2 + q^2))
//     (k_l + r_l = (p^2 + q^2)/(r_l - k_l), no cancellation where k_l < 0 < k_u; with both
//      offsets positive the plain ratio, with both at most zero the ratio of the r - k forms),
//   atan(u) - atan(v) = atan2(p q (k_u r_l - k_l r_u), p^2 r_u r_l + q^2 k_u k_l)
//     (u, v the two arguments: arg((1 + iu)(1 - iv)) with the factor p^2 r_u r_l > 0 taken out;
//      the difference lies in (-pi, pi), so the principal value is exact).
// Every log and arctangent of the 8 corners falls in exactly one (axis, corner) pair: 12
// logarithms and 12 two-argument arctangents instead of 24 and 24.
__host__ __device__ __forceinline__ double block_pair_term(double p, double q, double ku, double kl, double ru,
                                                           double rl) {
    // a vanishing p q drops the logarithm (its limit is 0; a charge on a face of a block with
    // K_k = 0 can make p, q or k_l zero).  The log's argument is formed without cancellation
    // wherever the point lies along the axis: below the box (k_l > 0) as (k_u + r_u)/(k_l + r_l),
    // above it (k_u <= 0) as (r_l - k_l)/(r_u - k_u), level with it as above.
    const double pq2 = p * p + q * q;
    double L = 0.0;
    if (p * q != 0.0) {
        const double arg = kl > 0.0 ? (ku + ru) / (kl + rl) : ku <= 0.0 ? (rl - kl) / (ru - ku) : (ku + ru) * (rl - kl) / pq2;
        L = p * q * log(arg);
    }
    const double A = 0.5 * p * p * atan2(p * q * (ku * rl - kl * ru), p * p * ru * rl + q * q * ku * kl);
    return L - A;
}

// Term j (0..11) of the regrouped corner sum: axis k = j / 4, the other two axes' corner from
// j % 4 (bit 0: p upper, bit 1: q upper), signed +1 when an even number of p, q is lower.
__host__ __device__ __forceinline__ double box_potential_paired_term(const double X[3], const double H[3], int j) {
    const int k = j >> 2, k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
    const double p = (j & 1) ? H[k1] - X[k1] : -H[k1] - X[k1];
    const double q = (j & 2) ? H[k2] - X[k2] : -H[k2] - X[k2];
    const double ku = H[k] - X[k], kl = -H[k] - X[k];
    const double pq2 = p * p + q * q;
    const double t = block_pair_term(p, q, ku, kl, sqrt(pq2 + ku * ku), sqrt(pq2 + kl * kl));
    const int lower = !(j & 1) + !(j & 2);
    return (lower & 1) ? -t : t;
}

// U(x) of the box [-H, H] at any point x: the 12 regrouped terms, the distances of the 8
// corners computed once.
__host__ __device__ __forceinline__ double box_potential_paired(const double X[3], const double H[3]) {
    const double lo[3] = {-H[0] - X[0], -H[1] - X[1], -H[2] - X[2]};
    const double up[3] = {H[0] - X[0], H[1] - X[1], H[2] - X[2]};
    double r[8];                          // corner c: bit k set = upper along axis k
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const double a = (c & 1) ? up[0] : lo[0], b = (c & 2) ? up[1] : lo[1], e = (c & 4) ? up[2] : lo[2];
        r[c] = sqrt(a * a + b * b + e * e);
    }
    double U = 0.0;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        const int k = j >> 2, k1 = k == 2 ? 0 : k + 1, k2 = k == 0 ? 2 : k - 1;
        const int cu = (1 << k) | ((j & 1) << k1) | (((j >> 1) & 1) << k2);   // upper along k
        const double t = block_pair_term((j & 1) ? up[k1] : lo[k1], (j & 2) ? up[k2] : lo[k2], up[k], lo[k], r[cu],
                                         r[cu & ~(1 << k)]);
        const int lower = !(j & 1) + !(j & 2);
        U += (lower & 1) ? -t : t;
    }
    return U;
}

}  // namespace psum
