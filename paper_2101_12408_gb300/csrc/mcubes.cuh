// Marching cubes for one cube of grid nodes (section "Surface Particle
// Sampling": the isocontour of the union-of-spheres level set, Chernyaev's
// marching cubes). No case table: each cube's crossing edges are joined into
// closed loops face by face, and each loop is cut into a fan of triangles.
//
// Corner c = x + 2 y + 4 z. Edge 4 a + j + 2 k runs along axis a between the two
// corners whose other two axes (in increasing order) have bits (j, k). Face
// f = 2 w + s lies at coordinate s along axis w; its corners are walked
// counter-clockwise as seen from outside the cube (in-face axes u = w + 1,
// v = w + 2 mod 3). Inside is phi < 0. Walking a face that way, a crossing edge
// is entering (outside corner to inside corner) or leaving, and every face
// segment runs from an entering crossing to a leaving one; each crossing edge is
// entering on exactly one of its two faces, so following the segments visits
// disjoint loops, oriented so that their triangles face outward. A face with
// four crossings is resolved by the asymptotic decider (the bilinear
// interpolant's saddle is inside when phi_a phi_c > phi_b phi_d for the inside
// diagonal a, c): joined, each entering crossing pairs with the leaving one
// before it, else with the one after it. The two cubes that share a face take
// the same decision from the same four values, so the surface is closed.
// Loops start at their smallest edge index; the fan of a loop with points
// p0..p(m-1) is (p0, pk, pk+1), k = 1..m-2; at most 10 triangles per cube.
//
// The header compiles as host C++ as well (a CPU test checks it against the
// FP64 oracle); on the device every product and sum is rounded on its own, and
// host builds must not contract them either (-ffp-contract=off).
#pragma once

#if defined(__CUDACC__)
#define MC_HD __host__ __device__ __forceinline__
#else
#define MC_HD inline
#endif

namespace mpm {
namespace mc {

MC_HD double rmul(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dmul_rn(a, b);
#else
    return a * b;
#endif
}
MC_HD double radd(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dadd_rn(a, b);
#else
    return a + b;
#endif
}
MC_HD double rsub(double a, double b) {
#if defined(__CUDA_ARCH__)
    return __dsub_rn(a, b);
#else
    return a - b;
#endif
}

// the two corners of edge e, lower index first
MC_HD void edge_corners(int e, int& c0, int& c1) {
    const int a = e >> 2, j = e & 1, k = (e >> 1) & 1;
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    c0 = (j << b) | (k << c);
    c1 = c0 | (1 << a);
}

// the edge joining adjacent corners ca, cb
MC_HD int edge_of(int ca, int cb) {
    const int lo = ca < cb ? ca : cb, d = ca ^ cb;
    const int a = d == 1 ? 0 : (d == 2 ? 1 : 2);
    const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
    return 4 * a + ((lo >> b) & 1) + 2 * ((lo >> c) & 1);
}

// corner k (0..3) of face f, counter-clockwise from outside
MC_HD int face_corner(int f, int k) {
    const int w = f >> 1, s = f & 1, u = (w + 1) % 3, v = (w + 2) % 3;
    // s = 1: (0,0) (1,0) (1,1) (0,1); s = 0: (0,0) (0,1) (1,1) (1,0)
    const int iu = s ? (k == 1 || k == 2) : (k >= 2);
    const int iv = s ? (k >= 2) : (k == 1 || k == 2);
    return (s << w) | (iu << u) | (iv << v);
}

struct Loops {
    signed char edge[12];   // the loops' edges, loop after loop
    signed char len[6];     // loop lengths
    int n;                  // number of loops
    int ntri;               // sum of (length - 2)
};

MC_HD void cube_loops(const double* cphi, Loops& L) {
    signed char nxt[12];
    for (int e = 0; e < 12; ++e) nxt[e] = -1;
    for (int f = 0; f < 6; ++f) {
        int fc[4];
        for (int k = 0; k < 4; ++k) fc[k] = face_corner(f, k);
        int ce[4], cent[4], nc = 0;
        for (int k = 0; k < 4; ++k) {
            const int a = fc[k], b = fc[(k + 1) & 3];
            const bool ia = cphi[a] < 0.0, ib = cphi[b] < 0.0;
            if (ia != ib) {
                ce[nc] = edge_of(a, b);
                cent[nc] = ib ? 1 : 0;
                ++nc;
            }
        }
        if (nc == 2) {
            const int ent = cent[0] ? ce[0] : ce[1];
            const int lea = cent[0] ? ce[1] : ce[0];
            nxt[ent] = (signed char)lea;
        } else if (nc == 4) {
            // corners alternate: the inside diagonal is (fc0, fc2) or (fc1, fc3)
            const int i0 = cphi[fc[0]] < 0.0 ? 0 : 1;
            const bool joined = rmul(cphi[fc[i0]], cphi[fc[i0 + 2]]) > rmul(cphi[fc[1 - i0]], cphi[fc[3 - i0]]);
            for (int k = 0; k < 4; ++k)
                if (cent[k]) nxt[ce[k]] = (signed char)(joined ? ce[(k + 3) & 3] : ce[(k + 1) & 3]);
        }
    }
    bool seen[12];
    for (int e = 0; e < 12; ++e) seen[e] = false;
    int total = 0;
    L.n = 0;
    L.ntri = 0;
    for (int e0 = 0; e0 < 12; ++e0) {
        if (nxt[e0] < 0 || seen[e0]) continue;
        int len = 0, e = e0;
        // bounded walk: at most 12 crossing edges, and a missing link ends it
        while (e >= 0 && !seen[e] && total + len < 12) {
            seen[e] = true;
            L.edge[total + len] = (signed char)e;
            ++len;
            e = nxt[e];
        }
        if (L.n < 6) {
            L.len[L.n++] = (signed char)len;
            total += len;
            if (len >= 3) L.ntri += len - 2;
        }
    }
}

// point on edge e: linear interpolation from its inside corner to its outside one
MC_HD void edge_point(const double* cphi, const int* q, double dx, const double* origin, int e, double* p) {
    int c0, c1;
    edge_corners(e, c0, c1);
    const int ci = cphi[c0] < 0.0 ? c0 : c1, co = ci == c0 ? c1 : c0;
    const double t = cphi[ci] / rsub(cphi[ci], cphi[co]);
    for (int a = 0; a < 3; ++a) {
        const double xa = radd(origin[a], rmul((double)(q[a] + ((ci >> a) & 1)) + 0.5, dx));
        const double xb = radd(origin[a], rmul((double)(q[a] + ((co >> a) & 1)) + 0.5, dx));
        p[a] = radd(xa, rmul(t, rsub(xb, xa)));
    }
}

// the cube's triangles: emit(t, p0, p1, p2) for t = 0..ntri-1; returns ntri
template <class Emit>
MC_HD int cube_triangles(const double* cphi, const int* q, double dx, const double* origin, Emit&& emit) {
    Loops L;
    cube_loops(cphi, L);
    int off = 0, t = 0;
    for (int l = 0; l < L.n; ++l) {
        const int m = L.len[l];
        if (m >= 3) {
            double p0[3], pa[3], pb[3];
            edge_point(cphi, q, dx, origin, L.edge[off], p0);
            edge_point(cphi, q, dx, origin, L.edge[off + 1], pb);
            for (int k = 1; k + 1 < m; ++k) {
                for (int a = 0; a < 3; ++a) pa[a] = pb[a];
                edge_point(cphi, q, dx, origin, L.edge[off + k + 1], pb);
                emit(t++, p0, pa, pb);
            }
        }
        off += m;
    }
    return t;
}

}  // namespace mc
}  // namespace mpm
