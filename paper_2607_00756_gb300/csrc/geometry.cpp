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
//    each parent's cell over the cell's area, from the parents' Delaunay
//    triangulation and the circumcentres of the triangles the query's
//    insertion removes (Watson's construction).
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

// ---- natural-neighbour (Sibson) coordinates from the Delaunay
// triangulation of the parents and the circumcentres of the triangles a
// query would destroy (Watson's construction): inserting q removes the
// triangles whose circumcircle holds it (the cavity); q's Voronoi cell is
// the polygon of the circumcentres of the new triangles (q, v_i, v_i+1)
// around the cavity boundary, and the part it takes from v_i's old cell is
// the convex polygon of the new circumcentres on either side of v_i and the
// circumcentres of the cavity triangles at v_i, in order around v_i.
//
// Positions are physical (x = h_x / l_x, y = h_y / l_y); orientation tests
// run exactly on the integer indices (scaling the axes keeps their sign),
// the in-circle test in FP64 with an error bound, within which the point is
// taken as on the circle (lattice points: exact zeros stay zero).

struct Node {
    int64_t ix, iy;     // integer beam index (h_x, h_y)
    double x, y;        // physical position
};

// > 0: c left of a -> b (counter-clockwise a, b, c), exact
int orient(const Node& a, const Node& b, const Node& c) {
    const int64_t v = (b.ix - a.ix) * (c.iy - a.iy) - (b.iy - a.iy) * (c.ix - a.ix);
    return (v > 0) - (v < 0);
}

// > 0: d strictly inside the circumcircle of the counter-clockwise triangle
// (a, b, c); 0 on it (within the FP64 error bound); < 0 outside
int incircle(const Node& a, const Node& b, const Node& c, const Node& d) {
    const double ax = a.x - d.x, ay = a.y - d.y, bx = b.x - d.x, by = b.y - d.y, cx = c.x - d.x, cy = c.y - d.y;
    const double al = ax * ax + ay * ay, bl = bx * bx + by * by, cl = cx * cx + cy * cy;
    const double t1 = al * (bx * cy - by * cx), t2 = bl * (cx * ay - cy * ax), t3 = cl * (ax * by - ay * bx);
    const double det = t1 + t2 + t3;
    const double perm = al * (std::fabs(bx * cy) + std::fabs(by * cx)) + bl * (std::fabs(cx * ay) + std::fabs(cy * ax)) +
                        cl * (std::fabs(ax * by) + std::fabs(ay * bx));
    if (std::fabs(det) <= 1e-12 * perm) return 0;
    return det > 0.0 ? 1 : -1;
}

struct Tri {
    int v[3];           // counter-clockwise
};

// centre of the circle through p, q, r, relative to the origin of (x, y)
void circumcentre(double px, double py, double qx, double qy, double rx, double ry, double& cx, double& cy) {
    const double ax = qx - px, ay = qy - py, bx = rx - px, by = ry - py;
    const double d = 2.0 * (ax * by - ay * bx);
    const double a2 = ax * ax + ay * ay, b2 = bx * bx + by * by;
    cx = px + (by * a2 - ay * b2) / d;
    cy = py + (ax * b2 - bx * a2) / d;
}

double polygon_area(const std::vector<double>& xs, const std::vector<double>& ys) {
    double s = 0.0;
    const size_t n = xs.size();
    for (size_t i = 0; i < n; ++i) {
        const size_t j = (i + 1) % n;
        s += xs[i] * ys[j] - xs[j] * ys[i];
    }
    return 0.5 * std::fabs(s);
}

// Delaunay triangulation by walking edges: every directed edge a -> b still
// open gets the triangle on its left whose circumcircle holds no other
// point (the candidate replaced only by a point strictly inside the current
// circle; among points on one circle any choice triangulates the empty
// polygon, since later edges only see points on their own left).
std::vector<Tri> delaunay(const std::vector<Node>& P) {
    const int n = (int)P.size();
    std::vector<Tri> tris;
    if (n < 3) return tris;
    // first hull edge: from the lowest point (then leftmost) to the point
    // with no other point strictly right of the edge, the nearest of any
    // collinear ones
    int a = 0;
    for (int i = 1; i < n; ++i)
        if (P[i].iy < P[a].iy || (P[i].iy == P[a].iy && P[i].ix < P[a].ix)) a = i;
    int b = -1;
    for (int i = 0; i < n; ++i) {
        if (i == a) continue;
        if (b < 0) { b = i; continue; }
        const int o = orient(P[a], P[b], P[i]);
        const auto d2 = [&](int k) { return (P[k].ix - P[a].ix) * (P[k].ix - P[a].ix) + (P[k].iy - P[a].iy) * (P[k].iy - P[a].iy); };
        if (o < 0 || (o == 0 && d2(i) < d2(b))) b = i;
    }
    std::set<std::pair<int, int>> done;
    std::vector<std::pair<int, int>> open{{a, b}};
    while (!open.empty()) {
        const auto e = open.back();
        open.pop_back();
        if (!done.insert(e).second) continue;
        int best = -1;
        for (int c = 0; c < n; ++c) {
            if (c == e.first || c == e.second || orient(P[e.first], P[e.second], P[c]) <= 0) continue;
            if (best < 0 || incircle(P[e.first], P[e.second], P[best], P[c]) > 0) best = c;
        }
        if (best < 0) continue;   // a hull edge: nothing on its left
        tris.push_back(Tri{{e.first, e.second, best}});
        done.insert({e.second, best});
        done.insert({best, e.first});
        // the neighbours across the two new edges lie on the left of their reverses
        open.push_back({best, e.second});
        open.push_back({e.first, best});
    }
    return tris;
}

}  // namespace

void bip_sibson_weights(const std::vector<int32_t>& parents, const std::vector<int32_t>& queries,
                        double ly, double lx, std::vector<double>& W) {
    const int np = (int)parents.size() / 2, nq = (int)queries.size() / 2;
    W.assign((size_t)nq * np, 0.0);
    if (np == 0) return;
    std::vector<Node> P(np);
    std::map<std::pair<int64_t, int64_t>, int> at;
    for (int i = 0; i < np; ++i) {
        P[i] = Node{parents[2 * i + 1], parents[2 * i], parents[2 * i + 1] / lx, parents[2 * i] / ly};
        at[{P[i].ix, P[i].iy}] = i;
    }
    const std::vector<Tri> T = delaunay(P);
    // hull edges: directed triangle edges (counter-clockwise) without the
    // reverse; with no triangle (collinear parents) the chain of consecutive
    // points along the line, both ways
    std::set<std::pair<int, int>> dir;
    for (const Tri& t : T)
        for (int k = 0; k < 3; ++k) dir.insert({t.v[k], t.v[(k + 1) % 3]});
    std::vector<std::pair<int, int>> hull;
    for (const auto& e : dir)
        if (!dir.count({e.second, e.first})) hull.push_back(e);
    if (T.empty() && np >= 2) {
        std::vector<int> ord(np);
        for (int i = 0; i < np; ++i) ord[i] = i;
        const double ux = P[np - 1].x - P[0].x, uy = P[np - 1].y - P[0].y;
        std::sort(ord.begin(), ord.end(), [&](int i, int j) { return P[i].x * ux + P[i].y * uy < P[j].x * ux + P[j].y * uy; });
        for (int i = 0; i + 1 < np; ++i) hull.push_back({ord[i], ord[i + 1]});
    }

    for (int qi = 0; qi < nq; ++qi) {
        double* w = &W[(size_t)qi * np];
        const Node q{queries[2 * qi + 1], queries[2 * qi], queries[2 * qi + 1] / lx, queries[2 * qi] / ly};
        auto it = at.find({q.ix, q.iy});
        if (it != at.end()) { w[it->second] = 1.0; continue; }
        if (np == 1) { w[0] = 1.0; continue; }
        // strictly inside the hull: strictly left of every hull edge
        bool inside = !T.empty();
        for (const auto& e : hull)
            if (inside && orient(P[e.first], P[e.second], q) <= 0) inside = false;
        if (!inside) {
            // on or outside the hull: the nearest hull edge's linear weights
            double best = INFINITY, bt = 0.0;
            int e0 = hull[0].first, e1 = hull[0].second;
            for (const auto& e : hull) {
                const Node &u = P[e.first], &v = P[e.second];
                const double dx = v.x - u.x, dy = v.y - u.y, dd = dx * dx + dy * dy;
                double t = ((q.x - u.x) * dx + (q.y - u.y) * dy) / dd;
                t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
                const double ex = q.x - (u.x + t * dx), ey = q.y - (u.y + t * dy), d = ex * ex + ey * ey;
                if (d < best) { best = d; bt = t; e0 = e.first; e1 = e.second; }
            }
            w[e0] += 1.0 - bt;
            w[e1] += bt;
            continue;
        }
        // the cavity: triangles whose circumcircle holds q strictly
        std::vector<int> cav;
        for (int t = 0; t < (int)T.size(); ++t)
            if (incircle(P[T[t].v[0]], P[T[t].v[1]], P[T[t].v[2]], q) > 0) cav.push_back(t);
        std::map<std::pair<int, int>, int> edge_tri;      // directed cavity edge -> its triangle
        for (int t : cav)
            for (int k = 0; k < 3; ++k) edge_tri[{T[t].v[k], T[t].v[(k + 1) % 3]}] = t;
        std::map<int, int> next;                          // boundary, counter-clockwise around q
        for (const auto& et : edge_tri)
            if (!edge_tri.count({et.first.second, et.first.first})) next[et.first.first] = et.first.second;
        std::vector<int> ring{next.begin()->first};
        while ((int)ring.size() <= (int)next.size()) {
            const int v = next[ring.back()];
            if (v == ring[0]) break;
            ring.push_back(v);
        }
        const int m = (int)ring.size();
        // circumcentres relative to q
        auto cc = [&](int i, int j, int k, bool with_q, double& cx, double& cy) {
            if (with_q)
                circumcentre(0.0, 0.0, P[i].x - q.x, P[i].y - q.y, P[j].x - q.x, P[j].y - q.y, cx, cy);
            else
                circumcentre(P[i].x - q.x, P[i].y - q.y, P[j].x - q.x, P[j].y - q.y, P[k].x - q.x, P[k].y - q.y, cx,
                             cy);
        };
        std::vector<double> stolen(m, 0.0);
        double total = 0.0;
        for (int i = 0; i < m; ++i) {
            const int vi = ring[i], vn = ring[(i + 1) % m], vp = ring[(i + m - 1) % m];
            std::vector<double> xs, ys;
            double cx, cy;
            cc(vi, vn, -1, true, cx, cy);
            xs.push_back(cx);
            ys.push_back(cy);
            // the cavity triangles at vi, counter-clockwise from the edge vi -> vn
            int a = vn;
            for (int guard = 0; guard <= (int)cav.size(); ++guard) {
                auto f = edge_tri.find({vi, a});
                if (f == edge_tri.end()) break;
                const Tri& t = T[f->second];
                int b = -1;
                for (int k = 0; k < 3; ++k)
                    if (t.v[k] == vi) b = t.v[(k + 2) % 3];
                cc(t.v[0], t.v[1], t.v[2], false, cx, cy);
                xs.push_back(cx);
                ys.push_back(cy);
                if (b == vp) break;
                a = b;
            }
            cc(vp, vi, -1, true, cx, cy);
            xs.push_back(cx);
            ys.push_back(cy);
            stolen[i] = polygon_area(xs, ys);
            total += stolen[i];
        }
        for (int i = 0; i < m; ++i) w[ring[i]] += stolen[i] / total;
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
    if (c.cube_ky > 0 && c.cube_kx > 0) {
        // a box of k-pixels centred on the zero beam, (h_y, h_x) ascending
        g.h_cube.clear();
        for (int a = -(c.cube_ky / 2); a < c.cube_ky - c.cube_ky / 2; ++a)
            for (int b = -(c.cube_kx / 2); b < c.cube_kx - c.cube_kx / 2; ++b) {
                g.h_cube.push_back(a);
                g.h_cube.push_back(b);
            }
    } else {
        g.h_cube = disc(c, g.lambda, c.theta_det, 1, 1);
    }
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
