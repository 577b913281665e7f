// Host-side FP64 construction of the per-pixel look-up tables of the coherent stage
// (Sec. II.C.1: HEALPix tiling, U and arrival-time tables; App. A Eqs. (strain_sngl),
// (svd)).  One epoch, Earth-fixed detectors.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <utility>
#include <vector>

#include "../../include/spiir.h"

namespace spiir {
int fail(int code, const char *fmt, ...);
void clear_error();
}  // namespace spiir

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr double kC = 299792458.0;  // m/s

struct Vec3 {
    double x, y, z;
};
inline double dot(const Vec3 &a, const Vec3 &b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// HEALPix pixel centres, RING order: rings north to south, increasing azimuth in a ring.
// Polar-cap ring at distance i from its pole: z = +-(1 - i^2/(3 ns^2)), 4i pixels at
// azimuth (j + 1/2) pi / (2i).  Belt ring i (ns <= i <= 3 ns from the north pole):
// z = 4/3 - 2i/(3 ns), 4 ns pixels at azimuth (j + s/2) pi / (2 ns), s = 1 if i - ns is
// even else 0.
void healpix_ring(int ns, std::vector<double> &theta, std::vector<double> &phi) {
    theta.clear();
    phi.clear();
    for (int i = 1; i <= 4 * ns - 1; ++i) {
        double z;
        int count;
        double ph0, dph;
        if (i < ns || i > 3 * ns) {
            const int q = (i < ns) ? i : 4 * ns - i;
            z = 1.0 - (double)q * q / (3.0 * ns * ns);
            if (i > 3 * ns) z = -z;
            count = 4 * q;
            dph = kPi / (2.0 * q);
            ph0 = 0.5 * dph;
        } else {
            z = 4.0 / 3.0 - 2.0 * i / (3.0 * ns);
            count = 4 * ns;
            dph = kPi / (2.0 * ns);
            ph0 = ((i - ns) % 2 == 0) ? 0.5 * dph : 0.0;
        }
        const double th = std::acos(z);
        for (int j = 0; j < count; ++j) {
            theta.push_back(th);
            phi.push_back(ph0 + j * dph);
        }
    }
}

}  // namespace

using namespace spiir;

extern "C" int spiir_sky_tables(int n_det, const double *pos, const double *arm_x, const double *arm_y,
                                const double *sigma, int nside, double rate, int32_t *delays, float *u_sig,
                                float *u_null) {
    clear_error();
    if (n_det < 2 || n_det > 4) return fail(SPIIR_EINVAL, "n_det = %d outside [2, 4]", n_det);
    if (nside < 1 || nside > 64) return fail(SPIIR_EINVAL, "nside = %d outside [1, 64]", nside);
    if (!(rate > 0) || !std::isfinite(rate)) return fail(SPIIR_EINVAL, "rate must be positive");
    if (!pos || !arm_x || !arm_y || !sigma || !delays || !u_sig || (n_det > 2 && !u_null))
        return fail(SPIIR_EINVAL, "NULL table pointer");
    std::vector<Vec3> r(n_det), X(n_det), Y(n_det);
    for (int d = 0; d < n_det; ++d) {
        r[d] = {pos[3 * d], pos[3 * d + 1], pos[3 * d + 2]};
        X[d] = {arm_x[3 * d], arm_x[3 * d + 1], arm_x[3 * d + 2]};
        Y[d] = {arm_y[3 * d], arm_y[3 * d + 1], arm_y[3 * d + 2]};
        for (double v : {r[d].x, r[d].y, r[d].z, X[d].x, X[d].y, X[d].z, Y[d].x, Y[d].y, Y[d].z, sigma[d]})
            if (!std::isfinite(v)) return fail(SPIIR_EINVAL, "non-finite geometry for detector %d", d);
        if (std::fabs(dot(X[d], X[d]) - 1) > 1e-6 || std::fabs(dot(Y[d], Y[d]) - 1) > 1e-6)
            return fail(SPIIR_EINVAL, "arm vectors of detector %d are not unit vectors", d);
        if (!(sigma[d] > 0)) return fail(SPIIR_EINVAL, "sigma[%d] must be positive", d);
    }
    std::vector<double> th, ph;
    healpix_ring(nside, th, ph);
    const int P = (int)th.size();
    for (int p = 0; p < P; ++p) {
        const double st = std::sin(th[p]), ct = std::cos(th[p]), sp = std::sin(ph[p]), cp = std::cos(ph[p]);
        const Vec3 nh{st * cp, st * sp, ct};
        const Vec3 ex{ct * cp, ct * sp, -st};  // e_theta
        const Vec3 ey{sp, -cp, 0.0};            // -e_phi
        // G_sigma rows: sigma_I (F+, Fx) with D = (X X^T - Y Y^T) / 2,
        // F+ = ex.D.ex - ey.D.ey, Fx = 2 ex.D.ey
        double G[4][2];
        for (int d = 0; d < n_det; ++d) {
            const double xa = dot(X[d], ex), xb = dot(X[d], ey), ya = dot(Y[d], ex), yb = dot(Y[d], ey);
            const double fp = 0.5 * ((xa * xa - ya * ya) - (xb * xb - yb * yb));
            const double fc = (xa * xb - ya * yb);
            G[d][0] = sigma[d] * fp;
            G[d][1] = sigma[d] * fc;
            const double v = -rate * dot(nh, r[d]) / kC;
            const long dl = std::lround(v);
            if (std::labs(dl) > 1024) return fail(SPIIR_EUNSUPPORTED, "arrival offset %ld too large", dl);
            delays[(int64_t)p * n_det + d] = (int32_t)dl;
        }
        // SVD of the n_det x 2 matrix through the symmetric eigenproblem of G^T G:
        // V rotates by angle a with tan(2a) = 2 m01 / (m00 - m11); U_s columns = G v_j / s_j.
        double m00 = 0, m01 = 0, m11 = 0;
        for (int d = 0; d < n_det; ++d) {
            m00 += G[d][0] * G[d][0];
            m01 += G[d][0] * G[d][1];
            m11 += G[d][1] * G[d][1];
        }
        const double ang = 0.5 * std::atan2(2.0 * m01, m00 - m11);
        const double c = std::cos(ang), s = std::sin(ang);
        double v[2][2] = {{c, s}, {-s, c}};
        double lam[2];
        for (int j = 0; j < 2; ++j)
            lam[j] = m00 * v[j][0] * v[j][0] + 2 * m01 * v[j][0] * v[j][1] + m11 * v[j][1] * v[j][1];
        if (lam[1] > lam[0]) {
            std::swap(lam[0], lam[1]);
            std::swap(v[0][0], v[1][0]);
            std::swap(v[0][1], v[1][1]);
        }
        double U[4][4] = {{0}};
        int ncol = 0;
        for (int j = 0; j < 2; ++j) {
            const bool keep = lam[0] > 0 && lam[j] > 1e-12 * lam[0];
            const double sv = keep ? std::sqrt(lam[j]) : 0.0;
            for (int d = 0; d < n_det; ++d) U[d][j] = keep ? (G[d][0] * v[j][0] + G[d][1] * v[j][1]) / sv : 0.0;
            if (keep) ++ncol;
        }
        // complete an orthonormal basis (modified Gram-Schmidt, two sweeps) for the null
        // space, starting from unit vectors
        int have = 2;
        for (int e = 0; e < n_det && have < n_det; ++e) {
            double w[4] = {0, 0, 0, 0};
            w[e] = 1.0;
            for (int sweep = 0; sweep < 2; ++sweep)
                for (int j = 0; j < have; ++j) {
                    double pr = 0;
                    for (int d = 0; d < n_det; ++d) pr += U[d][j] * w[d];
                    for (int d = 0; d < n_det; ++d) w[d] -= pr * U[d][j];
                }
            double nn = 0;
            for (int d = 0; d < n_det; ++d) nn += w[d] * w[d];
            nn = std::sqrt(nn);
            if (nn < 1e-6) continue;
            for (int d = 0; d < n_det; ++d) U[d][have] = w[d] / nn;
            ++have;
        }
        (void)ncol;
        for (int d = 0; d < n_det; ++d) {
            u_sig[((int64_t)p * n_det + d) * 2] = (float)U[d][0];
            u_sig[((int64_t)p * n_det + d) * 2 + 1] = (float)U[d][1];
            for (int j = 2; j < n_det; ++j)
                u_null[((int64_t)p * n_det + d) * (n_det - 2) + (j - 2)] = (float)U[d][j];
        }
    }
    return SPIIR_OK;
}
