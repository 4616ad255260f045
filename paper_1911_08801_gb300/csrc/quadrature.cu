// Icosahedron quadrature on the unit sphere (Sec. 3.3; the order-2 rule is printed in Appendix A).
//
// Order k: every face of the base solid carries a triangular lattice with k - 1 equal segments per
// edge; the lattice points are mapped to the sphere by central projection, and each point is
// weighted by the area of its spherical barycentric dual cell -- the region bounded by great-circle
// arcs through the centres of its neighbouring triangles and the midpoints of the edges between
// them, taken from the mapped points (or, with ASSN_ICO_FLAT_MIDPOINTS, from the flat lattice: the cell
// drawn on the flat face and mapped; the two agree at order 2).  N_q = 10 (k-1)^2 + 2.
//
// Base solid: twelve vertices joined as the 20 faces of the regular icosahedron.
// ASSN_ICO_REGULAR is the regular icosahedron (0, +-1, +-g), (+-1, +-g, 0), (+-g, 0, +-1) with
// g = (1 + sqrt 5)/2.  ASSN_ICO_PRINTED replaces each (+-g, 0, +-1) by the (+-1, 0, +-g) with the
// same signs, keeping the faces: on this solid the construction gives the paper's printed order-2
// points and weights.  Both are turned about the x axis so that (0, 1, g) maps to (0, 0, 1).
//
// Point numbering: the 12 vertices, then the interior points of the 30 edges (k - 2 each, counted
// from the lower-numbered end), then the interior points of the 20 faces ((k-2)(k-3)/2 each).  Every
// point is placed once from its barycentric definition, so points that faces share coincide exactly.
#include <math.h>

#include <vector>

#include "assn.h"
#include "problem.h"

namespace {

struct V3 {
    double x, y, z;
};

V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
V3 unit(V3 a) { return (1.0 / sqrt(dot(a, a))) * a; }

// Area of the spherical triangle with unit corners a, b, c: the solid-angle formula
// tan(E/2) = |a . (b x c)| / (1 + a.b + b.c + c.a) of Van Oosterom and Strackee (1983).
double sphere_area(V3 a, V3 b, V3 c) {
    return 2.0 * atan2(fabs(dot(a, cross(b, c))), 1.0 + dot(a, b) + dot(b, c) + dot(c, a));
}

struct Lattice {
    int n = 0;                   // segments per edge (order - 1)
    int face[20][3];             // vertex numbers, ascending
    int edge_of[12][12];         // edge number of a vertex pair, -1 if not joined
    int edge_end[30][2];         // the edge's vertices, ascending
    int count() const { return 10 * n * n + 2; }
    // Point with ca / n, cb / n, cc / n of the way to the face's vertices (ca + cb + cc = n).
    int node(int f, int ca, int cb, int cc) const {
        const int* v = face[f];
        if (ca == n) return v[0];
        if (cb == n) return v[1];
        if (cc == n) return v[2];
        if (ca == 0 || cb == 0 || cc == 0) {
            // on an edge: the two vertices with nonzero counts, ascending (faces list them so)
            const int u = ca ? v[0] : v[1], w = cc ? v[2] : v[1];
            const int cw = cc ? cc : cb;
            return 12 + edge_of[u][w] * (n - 1) + (cw - 1);
        }
        const int first = 12 + 30 * (n - 1) + f * ((n - 1) * (n - 2) / 2);
        return first + (cb - 1) * (n - 1) - (cb - 1) * cb / 2 + (cc - 1);
    }
};

}  // namespace

extern "C" int assn_icosahedron_quadrature(int order, int base, double* omega, double* w, int capacity) {
    if (order < 2 || order > ASSN_ICO_MAX_ORDER) return ASSN_ERR_ARG;
    if ((base & ~(ASSN_ICO_REGULAR | ASSN_ICO_FLAT_MIDPOINTS)) != 0) return ASSN_ERR_ARG;
    const bool regular = (base & ASSN_ICO_REGULAR) != 0, flat_mid = (base & ASSN_ICO_FLAT_MIDPOINTS) != 0;
    Lattice L;
    L.n = order - 1;
    const int N = L.count();
    if (!omega || !w) return N;
    if (capacity < N) return ASSN_ERR_ARG;

    const double g = 0.5 * (1.0 + sqrt(5.0));
    V3 reg[12], vert[12];
    int m = 0;
    for (int group = 0; group < 3; ++group)
        for (int s = 0; s < 4; ++s, ++m) {
            const double a = (s & 1) ? -1.0 : 1.0, b = (s & 2) ? -g : g;
            if (group == 0) reg[m] = vert[m] = {0.0, a, b};
            if (group == 1) reg[m] = vert[m] = {a, b, 0.0};
            if (group == 2) {
                reg[m] = {b, 0.0, a};   // (+-g, 0, +-1); the printed base puts (+-1, 0, +-g), same signs, here
                vert[m] = regular ? reg[m] : V3{b / g, 0.0, a * g};
            }
        }
    // joins of the regular icosahedron: vertex pairs at distance 2
    int ne = 0;
    for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
            L.edge_of[i][j] = -1;
            if (j > i && fabs(dot(reg[i] - reg[j], reg[i] - reg[j]) - 4.0) < 1e-9) {
                L.edge_end[ne][0] = i;
                L.edge_end[ne][1] = j;
                L.edge_of[i][j] = ne++;
            }
        }
    int nf = 0;
    for (int i = 0; i < 12; ++i)
        for (int j = i + 1; j < 12; ++j)
            for (int k = j + 1; k < 12; ++k)
                if (L.edge_of[i][j] >= 0 && L.edge_of[j][k] >= 0 && L.edge_of[i][k] >= 0) {
                    L.face[nf][0] = i;
                    L.face[nf][1] = j;
                    L.face[nf][2] = k;
                    ++nf;
                }
    if (ne != 30 || nf != 20) return ASSN_ERR_STATE;   // cannot happen: the solid is fixed

    // turn about x by atan(1/g): (0, 1, g) -> (0, 0, |.|)
    const double ca = g / sqrt(1.0 + g * g), sa = 1.0 / sqrt(1.0 + g * g);
    for (auto& v : vert) v = {v.x, ca * v.y - sa * v.z, sa * v.y + ca * v.z};

    const int n = L.n;
    std::vector<V3> F(N);                               // the flat lattice points
    for (int i = 0; i < 12; ++i) F[i] = vert[i];
    for (int e = 0; e < 30; ++e)
        for (int t = 1; t < n; ++t) {
            const V3 a = vert[L.edge_end[e][0]], b = vert[L.edge_end[e][1]];
            F[12 + e * (n - 1) + t - 1] = a + ((double)t / n) * (b - a);
        }
    for (int f = 0; f < 20; ++f)
        for (int cb = 1; cb < n; ++cb)
            for (int cc = 1; cb + cc < n; ++cc) {
                const V3 a = vert[L.face[f][0]], b = vert[L.face[f][1]], c = vert[L.face[f][2]];
                F[L.node(f, n - cb - cc, cb, cc)] = a + ((double)cb / n) * (b - a) + ((double)cc / n) * (c - a);
            }
    std::vector<V3> P(N);                               // mapped to the sphere
    for (int i = 0; i < N; ++i) P[i] = unit(F[i]);
    const std::vector<V3>& M = flat_mid ? F : P;        // the points the cells' midpoints come from

    std::vector<double> W(N, 0.0);
    auto add_triangle = [&](int i0, int i1, int i2) {
        const int id[3] = {i0, i1, i2};
        const V3 c = unit(M[i0] + M[i1] + M[i2]);
        for (int k = 0; k < 3; ++k) {
            const V3 a = M[id[k]], b = M[id[(k + 1) % 3]], d = M[id[(k + 2) % 3]];
            W[id[k]] += sphere_area(P[id[k]], unit(a + b), c) + sphere_area(P[id[k]], c, unit(a + d));
        }
    };
    for (int f = 0; f < 20; ++f)
        for (int cb = 0; cb < n; ++cb)
            for (int cc = 0; cb + cc < n; ++cc) {
                const int r = n - cb - cc;
                add_triangle(L.node(f, r, cb, cc), L.node(f, r - 1, cb + 1, cc), L.node(f, r - 1, cb, cc + 1));
                if (cb + cc + 2 <= n)
                    add_triangle(L.node(f, r - 1, cb + 1, cc), L.node(f, r - 2, cb + 1, cc + 1),
                                 L.node(f, r - 1, cb, cc + 1));
            }
    for (int q = 0; q < N; ++q) {
        omega[3 * q] = P[q].x;
        omega[3 * q + 1] = P[q].y;
        omega[3 * q + 2] = P[q].z;
        w[q] = W[q];
    }
    return N;
}

extern "C" int assn_set_icosahedron_quadrature(assn_problem* p, int order, int base) {
    if (!p) return ASSN_ERR_ARG;
    if (order < 2 || 10 * (order - 1) * (order - 1) + 2 > ASSN_MAX_Q)
        return assn::problem_fail(p, ASSN_ERR_ARG, "icosahedron order out of range (2 .. 11 for Q <= 1024)");
    if ((base & ~(ASSN_ICO_REGULAR | ASSN_ICO_FLAT_MIDPOINTS)) != 0)
        return assn::problem_fail(p, ASSN_ERR_ARG, "unknown icosahedron base");
    const int N = 10 * (order - 1) * (order - 1) + 2;
    std::vector<double> om(3 * (size_t)N), w(N);
    const int r = assn_icosahedron_quadrature(order, base, om.data(), w.data(), N);
    if (r != N) return assn::problem_fail(p, r < 0 ? r : ASSN_ERR_STATE, "icosahedron quadrature failed");
    return assn_set_quadrature(p, N, om.data(), w.data());
}
