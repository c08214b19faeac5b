// Host geometry of the BiP-PRISM map in FP64: beams, PRISM subsampling,
// hex-ring parents and Sibson natural-neighbour weights.
//
//  * aperture beams {h : |q| lambda <= alpha}, kept when h = 0 mod f
//    (Sec. 2.1; Algorithm 2 build step; Sec. 2.2.2 beam subsampling);
//  * detector beams |q| lambda <= theta_det, PRISM-subsampled by (dfy, dfx)
//    (Algorithm 4; qEELS wants the resolved axis at 1, Sec. 2.2.6), and the
//    cube's complete basis, the same disc unsubsampled (Sec. 2.2.6);
//  * hex-ring parents: DC plus n_radial rings with n_angular (1 + i) samples
//    on ring i, snapped to the nearest beam, deduplicated (Sec. 2.2.3);
//  * Sibson weights (Eq. nnw): the area the query's Voronoi cell takes from
//    each parent's cell over the cell's area, by half-plane clipping.
//
// Readings where the paper is silent: beams sorted by (h_y, h_x); aperture
// edge inclusive with 1e-12 relative slack; ring radius R (i+1)/n_radial
// with R the largest retained |q|; angles 2 pi k/(n_angular (1+i)) from
// +q_x towards +q_y; snapping ties (relative 1e-9) to the smallest
// (h_y, h_x); a query on or outside the parents' convex hull takes the
// linear weights of the nearest hull edge's end points.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <utility>

#include "bip_internal.h"

namespace {

constexpr double kM0C2 = 510998.95;             // eV
constexpr double kHC = 12398.419843320026;      // eV * Angstrom
constexpr double kPi = 3.14159265358979323846;

int signed_bin(int k, int n) { return k < (n + 1) / 2 ? k : k - n; }

// beams of the disc |q| lambda <= angle with h = 0 mod f, sorted (h_y, h_x)
std::vector<int32_t> disc(const bip_config& c, double lam, double angle, int fy, int fx) {
    std::vector<int> hy, hx;
    for (int k = 0; k < c.ny; ++k) hy.push_back(signed_bin(k, c.ny));
    for (int k = 0; k < c.nx; ++k) hx.push_back(signed_bin(k, c.nx));
    std::sort(hy.begin(), hy.end());
    std::sort(hx.begin(), hx.end());
    std::vector<int32_t> out;
    for (int a : hy) {
        if (a % fy != 0) continue;
        for (int b : hx) {
            if (b % fx != 0) continue;
            double qy = a / c.ly, qx = b / c.lx;
            double q = std::sqrt(qy * qy + qx * qx);
            if (q * lam <= angle * (1.0 + 1e-12)) {
                out.push_back(a);
                out.push_back(b);
            }
        }
    }
    return out;
}

std::vector<int32_t> hex_ring(const std::vector<int32_t>& h, double ly, double lx, int nrad, int nang) {
    const int n = (int)h.size() / 2;
    std::vector<double> qy(n), qx(n);
    double R = 0.0;
    for (int i = 0; i < n; ++i) {
        qy[i] = h[2 * i] / ly;
        qx[i] = h[2 * i + 1] / lx;
        R = std::max(R, std::sqrt(qy[i] * qy[i] + qx[i] * qx[i]));
    }
    std::vector<std::pair<double, double>> targets{{0.0, 0.0}};
    for (int i = 0; i < nrad; ++i) {
        double r = R * (i + 1) / nrad;
        int m = nang * (1 + i);
        for (int k = 0; k < m; ++k) {
            double th = 2.0 * kPi * k / m;
            targets.push_back({r * std::sin(th), r * std::cos(th)});
        }
    }
    std::vector<int32_t> chosen;
    for (auto& t : targets) {
        double best = INFINITY;
        for (int i = 0; i < n; ++i) {
            double dy = qy[i] - t.first, dx = qx[i] - t.second;
            best = std::min(best, dy * dy + dx * dx);
        }
        int pick = -1;
        for (int i = 0; i < n; ++i) {
            double dy = qy[i] - t.first, dx = qx[i] - t.second;
            if (dy * dy + dx * dx <= best * (1.0 + 1e-9)) {
                if (pick < 0 || h[2 * i] < h[2 * pick] ||
                    (h[2 * i] == h[2 * pick] && h[2 * i + 1] < h[2 * pick + 1]))
                    pick = i;
            }
        }
        if (pick >= 0 && std::find(chosen.begin(), chosen.end(), pick) == chosen.end())
            chosen.push_back(pick);
    }
    return chosen;
}

// ---- convex polygons in relative physical coordinates
using Pt = std::pair<double, double>;   // (y, x)

std::vector<Pt> clip(const std::vector<Pt>& poly, double a0, double a1, double c) {
    std::vector<Pt> out;
    const size_t n = poly.size();
    out.reserve(n + 2);
    for (size_t i = 0; i < n; ++i) {
        const Pt& p = poly[i];
        const Pt& q = poly[(i + 1) % n];
        double fp = a0 * p.first + a1 * p.second - c;
        double fq = a0 * q.first + a1 * q.second - c;
        if (fp <= 0.0) out.push_back(p);
        if ((fp < 0.0 && fq > 0.0) || (fq < 0.0 && fp > 0.0)) {
            double t = fp / (fp - fq);
            out.push_back({p.first + t * (q.first - p.first), p.second + t * (q.second - p.second)});
        }
    }
    return out;
}

double area(const std::vector<Pt>& poly) {
    if (poly.size() < 3) return 0.0;
    double s = 0.0;
    for (size_t i = 0; i < poly.size(); ++i) {
        const Pt& a = poly[i];
        const Pt& b = poly[(i + 1) % poly.size()];
        s += a.second * b.first - b.second * a.first;
    }
    return 0.5 * std::fabs(s);
}

using IPt = std::pair<int64_t, int64_t>;

int64_t cross(const IPt& o, const IPt& a, const IPt& b) {
    return (a.first - o.first) * (b.second - o.second) - (a.second - o.second) * (b.first - o.first);
}

// convex hull keeping collinear boundary points (monotone chain)
std::vector<IPt> hull(std::vector<IPt> P) {
    std::sort(P.begin(), P.end());
    P.erase(std::unique(P.begin(), P.end()), P.end());
    if (P.size() <= 2) return P;
    std::vector<IPt> lo, up;
    for (auto& p : P) {
        while (lo.size() >= 2 && cross(lo[lo.size() - 2], lo.back(), p) < 0) lo.pop_back();
        lo.push_back(p);
    }
    for (auto it = P.rbegin(); it != P.rend(); ++it) {
        while (up.size() >= 2 && cross(up[up.size() - 2], up.back(), *it) < 0) up.pop_back();
        up.push_back(*it);
    }
    std::vector<IPt> h(lo.begin(), lo.end() - 1);
    h.insert(h.end(), up.begin(), up.end() - 1);
    std::vector<IPt> out;
    std::set<IPt> seen;
    for (auto& p : h)
        if (seen.insert(p).second) out.push_back(p);
    return out;
}

bool strictly_inside(const std::vector<IPt>& H, const IPt& q) {
    const size_t n = H.size();
    if (n < 3) return false;
    int64_t s = 0;
    for (size_t i = 0; i < n; ++i) s += cross({0, 0}, H[i], H[(i + 1) % n]);
    const int orient = s > 0 ? 1 : -1;
    for (size_t i = 0; i < n; ++i) {
        int64_t c = cross(H[i], H[(i + 1) % n], q);
        if (c * orient <= 0) return false;
    }
    return true;
}

}  // namespace

void bip_sibson_weights(const std::vector<int32_t>& parents, const std::vector<int32_t>& queries,
                        double ly, double lx, std::vector<double>& W) {
    const int np = (int)parents.size() / 2, nq = (int)queries.size() / 2;
    W.assign((size_t)nq * np, 0.0);
    if (np == 0) return;
    std::vector<double> py(np), px(np);
    std::map<IPt, int> lut;
    std::vector<IPt> pts;
    for (int i = 0; i < np; ++i) {
        py[i] = parents[2 * i] / ly;
        px[i] = parents[2 * i + 1] / lx;
        IPt ip{parents[2 * i], parents[2 * i + 1]};
        lut[ip] = i;
        pts.push_back(ip);
    }
    const std::vector<IPt> H = hull(pts);
    std::vector<int> hidx;
    for (auto& p : H) hidx.push_back(lut[p]);

    for (int b = 0; b < nq; ++b) {
        double* w = &W[(size_t)b * np];
        IPt hb{queries[2 * b], queries[2 * b + 1]};
        auto it = lut.find(hb);
        if (it != lut.end()) { w[it->second] = 1.0; continue; }
        if (np == 1) { w[0] = 1.0; continue; }
        const double qy = hb.first / ly, qx = hb.second / lx;
        if (!strictly_inside(H, hb)) {
            // nearest hull edge, linear weights of its end points
            double best = INFINITY, bt = 0.0;
            int be = 0;
            const int nh = (int)hidx.size();
            for (int e = 0; e < nh; ++e) {
                int i0 = hidx[e], i1 = hidx[(e + 1) % nh];
                double dy = py[i1] - py[i0], dx = px[i1] - px[i0];
                double dd = dy * dy + dx * dx;
                double t = dd == 0.0 ? 0.0 : ((qy - py[i0]) * dy + (qx - px[i0]) * dx) / dd;
                t = std::min(1.0, std::max(0.0, t));
                double ey = qy - (py[i0] + t * dy), ex = qx - (px[i0] + t * dx);
                double d = ey * ey + ex * ex;
                if (d < best) { best = d; be = e; bt = t; }
            }
            w[hidx[be]] += 1.0 - bt;
            w[hidx[(be + 1) % nh]] += bt;
            continue;
        }
        // interior: Voronoi cell of the query against all parents
        std::vector<double> ry(np), rx(np), dist(np);
        for (int i = 0; i < np; ++i) {
            ry[i] = py[i] - qy;
            rx[i] = px[i] - qx;
            dist[i] = std::sqrt(ry[i] * ry[i] + rx[i] * rx[i]);
        }
        std::vector<int> order(np);
        for (int i = 0; i < np; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return dist[a] < dist[c]; });
        double box = 4.0 * *std::max_element(dist.begin(), dist.end());
        std::vector<Pt> cell;
        for (;;) {
            cell = {{-box, -box}, {-box, box}, {box, box}, {box, -box}};
            for (int j : order) {
                cell = clip(cell, 2.0 * ry[j], 2.0 * rx[j], ry[j] * ry[j] + rx[j] * rx[j]);
                if (cell.empty()) break;
            }
            double rmax = 0.0;
            for (auto& p : cell) rmax = std::max(rmax, std::max(std::fabs(p.first), std::fabs(p.second)));
            if (rmax < box * (1.0 - 1e-9)) break;
            box *= 4.0;
        }
        const double a_new = area(cell);
        double r_new = 0.0;
        for (auto& p : cell) r_new = std::max(r_new, std::hypot(p.first, p.second));
        const double lim = 2.0 * r_new + dist[order[0]] + 1e-12 * r_new;
        std::vector<int> cand;
        for (int j : order)
            if (dist[j] <= lim) cand.push_back(j);
        for (int p : cand) {
            std::vector<Pt> piece = cell;
            for (int j : cand) {
                if (j == p) continue;
                piece = clip(piece, 2.0 * (ry[j] - ry[p]), 2.0 * (rx[j] - rx[p]),
                             (ry[j] * ry[j] + rx[j] * rx[j]) - (ry[p] * ry[p] + rx[p] * rx[p]));
                if (piece.empty()) break;
            }
            w[p] = area(piece) / a_new;
        }
    }
}

void bip_aberration_phase(const bip_config& c, double lambda, int hy, int hx, double* chi, double* d_defocus,
                          double* d_cs) {
    const double q2 = (hy / c.ly) * (hy / c.ly) + (hx / c.lx) * (hx / c.lx);
    const double l3 = lambda * lambda * lambda;
    if (chi) *chi = kPi * lambda * c.defocus * q2 + 0.5 * kPi * c.cs * l3 * q2 * q2;
    if (d_defocus) *d_defocus = kPi * lambda * q2;
    if (d_cs) *d_cs = 0.5 * kPi * l3 * q2 * q2;
}

void bip_set_psi(const bip_config& c, BipGeometry& g) {
    g.psi_beam.resize(g.B);
    for (int b = 0; b < g.B; ++b) {
        double x = 0.0;
        bip_aberration_phase(c, g.lambda, g.h_beam[2 * b], g.h_beam[2 * b + 1], &x, nullptr, nullptr);
        g.psi_beam[b] = std::complex<double>(std::cos(x), -std::sin(x));
    }
}

bip_status bip_build_geometry(const bip_config& c, BipGeometry& g, std::string& err) {
    g.lambda = kHC / std::sqrt(c.e0 * (2.0 * kM0C2 + c.e0));
    g.sigma = (2.0 * kPi / (g.lambda * c.e0)) * (kM0C2 + c.e0) / (2.0 * kM0C2 + c.e0);
    // the discs must fit inside the grid's Nyquist band
    const double qmax_grid = std::min(c.ny / (2.0 * c.ly), c.nx / (2.0 * c.lx));
    if (c.alpha / g.lambda >= qmax_grid || c.theta_det / g.lambda >= qmax_grid) {
        err = "aperture or detector disc exceeds the grid's Nyquist band";
        return BIP_ERR_SHAPE;
    }
    std::vector<int32_t> full = disc(c, g.lambda, c.alpha, 1, 1);
    g.n_full = (int)full.size() / 2;
    g.h_beam = disc(c, g.lambda, c.alpha, c.fy, c.fx);
    g.dfy = c.dfy > 0 ? c.dfy : c.fy;
    g.dfx = c.dfx > 0 ? c.dfx : c.fx;
    g.h_det = disc(c, g.lambda, c.theta_det, g.dfy, g.dfx);
    g.h_cube = disc(c, g.lambda, c.theta_det, 1, 1);
    g.B = (int)g.h_beam.size() / 2;
    g.n_det = (int)g.h_det.size() / 2;
    g.n_cube = (int)g.h_cube.size() / 2;
    if (g.B == 0 || g.n_det == 0) {
        err = "empty aperture or detector beam set";
        return BIP_ERR_SHAPE;
    }
    double s = 0.0;
    for (int i = 0; i < g.n_full; ++i) s += 1.0;   // |Psi| = 1 inside the aperture
    g.psi_norm = std::sqrt((double)c.ny * c.nx * s);
    bip_set_psi(c, g);
    g.p1 = hex_ring(g.h_beam, c.ly, c.lx, c.nrad1, c.nang1);
    g.p2 = hex_ring(g.h_det, c.ly, c.lx, c.nrad2, c.nang2);
    g.Bp1 = (int)g.p1.size();
    g.Bp2 = (int)g.p2.size();
    std::vector<int32_t> hp1, hp2;
    for (int p : g.p1) { hp1.push_back(g.h_beam[2 * p]); hp1.push_back(g.h_beam[2 * p + 1]); }
    for (int p : g.p2) { hp2.push_back(g.h_det[2 * p]); hp2.push_back(g.h_det[2 * p + 1]); }
    bip_sibson_weights(hp1, g.h_beam, c.ly, c.lx, g.w1);
    bip_sibson_weights(hp2, g.h_det, c.ly, c.lx, g.w2);
    return BIP_OK;
}
