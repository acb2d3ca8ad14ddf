/*
 * Oracle (test infrastructure only): generalized Newell demagnetization tensor,
 * written out exactly as the paper derives it, for one real type.
 *
 * This file is included twice by newell.c, once with REAL = double (suffix _d)
 * and once with REAL = _Float128 (suffix _q).  The macros RSQRT, RASINH, RATAN,
 * RPI and SFX are supplied by the includer.
 *
 * Notation follows Sec. 2 of the paper: the target cuboid tau has dimensions
 * (tx, ty, tz) = (Delta x, Delta y, Delta z), the source cuboid tau' has
 * dimensions (sx, sy, sz) = (Delta x', Delta y', Delta z'); the source occupies
 * [0,sx]x[0,sy]x[0,sz] and the target [X,X+tx]x[Y,Y+ty]x[Z,Z+tz], so (X,Y,Z)
 * is the target corner minus the source corner.  The tensor is normalised by
 * the target volume |tau| = tx*ty*tz (Sec. 2, Eq. Nxx and Eq. Nxy).
 *
 * Only tests, __graft_entry__.smoke() and bench.py's CPU baseline may use this.
 */

#define CAT2(a, b) a##b
#define CAT(a, b) CAT2(a, b)
#define FN(name) CAT(name, SFX)

/* Newell f (Sec. 2.1): the indefinite integral whose mixed derivative
 * d^2/dy^2 d^2/dz^2 f equals 1/sqrt(x^2+y^2+z^2).  Each product whose
 * prefactor vanishes is taken at its limit, zero (0*asinh(./0), 0*atan(./0)). */
static REAL FN(newell_f)(REAL x, REAL y, REAL z)
{
    REAL x2 = x * x, y2 = y * y, z2 = z * z;
    REAL R = RSQRT(x2 + y2 + z2);
    REAL res = (2 * x2 - y2 - z2) * R / 6;
    if (y != 0 && (x2 + z2) > 0)
        res += y / 2 * (z2 - x2) * RASINH(y / RSQRT(x2 + z2));
    if (z != 0 && (x2 + y2) > 0)
        res += z / 2 * (y2 - x2) * RASINH(z / RSQRT(x2 + y2));
    if (x != 0 && y != 0 && z != 0)
        res -= x * y * z * RATAN(y * z / (x * R));
    return res;
}

/* Newell g (Sec. 2.2): the indefinite integral with d/dx d/dy d^2/dz^2 g =
 * 1/sqrt(x^2+y^2+z^2).  Vanishing prefactors again give zero terms. */
static REAL FN(newell_g)(REAL x, REAL y, REAL z)
{
    REAL x2 = x * x, y2 = y * y, z2 = z * z;
    REAL R = RSQRT(x2 + y2 + z2);
    REAL res = -x * y * R / 3;
    if (x != 0 && y != 0 && z != 0)
        res += x * y * z * RASINH(z / RSQRT(x2 + y2));
    if (y != 0)
        res += y / 6 * (3 * z2 - y2) * RASINH(x / RSQRT(y2 + z2));
    if (x != 0)
        res += x / 6 * (3 * z2 - x2) * RASINH(y / RSQRT(x2 + z2));
    if (z != 0 && x != 0 && y != 0)
        res -= z2 * z / 6 * RATAN(x * y / (z * R));
    if (y != 0 && x != 0 && z != 0)
        res -= z * y2 / 2 * RATAN(x * z / (y * R));
    if (x != 0 && y != 0 && z != 0)
        res -= z * x2 / 2 * RATAN(y * z / (x * R));
    return res;
}

/* ---- N_xx (Sec. 2.1, Eq. Nxx, Eq. F, App. A) ---------------------------- */

/* F_2 (Eq. F2 / Eq. F_2).  full=1 keeps all four f terms of Eq. F_2; full=0
 * keeps only f(X,Y,Z): the other three are constant in Y or in Z and cancel in
 * the weighted sums of F_1 and F, which is the 256 -> 64 term reduction stated
 * at the end of Sec. 2.1. */
static REAL FN(F2)(REAL X, REAL Y, REAL Z, int full)
{
    REAL v = FN(newell_f)(X, Y, Z);
    if (full)
        v += -FN(newell_f)(X, 0, Z) - FN(newell_f)(X, Y, 0) + FN(newell_f)(X, 0, 0);
    return v;
}

/* F_1 (App. A): groups the four y-offsets of the source and target faces. */
static REAL FN(F1)(REAL X, REAL Y, REAL Z, REAL ty, REAL sy, int full)
{
    return FN(F2)(X, Y + ty, Z, full) - FN(F2)(X, Y, Z, full)
         - FN(F2)(X, Y + ty - sy, Z, full) + FN(F2)(X, Y - sy, Z, full);
}

/* F (App. A): the parallel-face interaction of Eq. F as four F_1 terms in z. */
static REAL FN(Fface)(REAL X, REAL Y, REAL Z, REAL ty, REAL tz, REAL sy, REAL sz, int full)
{
    return FN(F1)(X, Y, Z + tz, ty, sy, full) - FN(F1)(X, Y, Z, ty, sy, full)
         - FN(F1)(X, Y, Z + tz - sz, ty, sy, full) + FN(F1)(X, Y, Z - sz, ty, sy, full);
}

/* Generalized N_xx (Eq. Nxx): the four x-face pairs of target and source. */
static REAL FN(gen_nxx)(REAL X, REAL Y, REAL Z, const REAL t[3], const REAL s[3], int full)
{
    REAL acc = FN(Fface)(X, Y, Z, t[1], t[2], s[1], s[2], full)
             - FN(Fface)(X + t[0], Y, Z, t[1], t[2], s[1], s[2], full)
             - FN(Fface)(X - s[0], Y, Z, t[1], t[2], s[1], s[2], full)
             + FN(Fface)(X + t[0] - s[0], Y, Z, t[1], t[2], s[1], s[2], full);
    return acc / (4 * RPI * t[0] * t[1] * t[2]);
}

/* ---- N_xy (Sec. 2.2, Eq. Nxy, Eq. G, App. B) ---------------------------- */

/* G_2 (Eq. G2_as_g).  full=0 drops g(X,Y,0), which is constant in Z and
 * cancels in G_1 (the 128 -> 64 term reduction stated at the end of Sec. 2.2). */
static REAL FN(G2)(REAL X, REAL Y, REAL Z, int full)
{
    REAL v = FN(newell_g)(X, Y, Z);
    if (full)
        v -= FN(newell_g)(X, Y, 0);
    return v;
}

/* G_1 (App. B): four z offsets. */
static REAL FN(G1)(REAL X, REAL Y, REAL Z, REAL tz, REAL sz, int full)
{
    return FN(G2)(X, Y, Z + tz, full) - FN(G2)(X, Y, Z, full)
         - FN(G2)(X, Y, Z + tz - sz, full) + FN(G2)(X, Y, Z - sz, full);
}

/* G (App. B): four offsets in x (target extent) and y (source extent). */
static REAL FN(Gface)(REAL X, REAL Y, REAL Z, REAL tx, REAL tz, REAL sy, REAL sz, int full)
{
    return FN(G1)(X + tx, Y, Z, tz, sz, full) - FN(G1)(X + tx, Y - sy, Z, tz, sz, full)
         - FN(G1)(X, Y, Z, tz, sz, full) + FN(G1)(X, Y - sy, Z, tz, sz, full);
}

/* Generalized N_xy (Eq. Nxy).  The fourth term is taken as G(X - Delta x',
 * Y + Delta y, Z): the printed "Y - Delta y" contradicts the face geometry
 * (target y-faces at Y and Y + Delta y) and fails the dipole limit. */
static REAL FN(gen_nxy)(REAL X, REAL Y, REAL Z, const REAL t[3], const REAL s[3], int full)
{
    REAL acc = FN(Gface)(X, Y, Z, t[0], t[2], s[1], s[2], full)
             - FN(Gface)(X - s[0], Y, Z, t[0], t[2], s[1], s[2], full)
             - FN(Gface)(X, Y + t[1], Z, t[0], t[2], s[1], s[2], full)
             + FN(Gface)(X - s[0], Y + t[1], Z, t[0], t[2], s[1], s[2], full);
    return acc / (4 * RPI * t[0] * t[1] * t[2]);
}

/* All six components by permutation of the axes (Sec. 2, after Eq. N):
 *   N_yy = N_xx with x<->y, N_zz = N_xx with x<->z,
 *   N_xz = N_xy with y<->z, N_yz = N_zy = N_xy with x<->z.
 * out = {xx, yy, zz, xy, xz, yz}. */
static void FN(gen_tensor)(REAL X, REAL Y, REAL Z, const REAL t[3], const REAL s[3],
                           int full, REAL out[6])
{
    REAL tyx[3] = {t[1], t[0], t[2]}, syx[3] = {s[1], s[0], s[2]};
    REAL tzx[3] = {t[2], t[1], t[0]}, szx[3] = {s[2], s[1], s[0]};
    REAL tzy[3] = {t[0], t[2], t[1]}, szy[3] = {s[0], s[2], s[1]};
    out[0] = FN(gen_nxx)(X, Y, Z, t, s, full);
    out[1] = FN(gen_nxx)(Y, X, Z, tyx, syx, full);
    out[2] = FN(gen_nxx)(Z, Y, X, tzx, szx, full);
    out[3] = FN(gen_nxy)(X, Y, Z, t, s, full);
    out[4] = FN(gen_nxy)(X, Z, Y, tzy, szy, full);
    out[5] = FN(gen_nxy)(Z, Y, X, tzx, szx, full);
}

#undef FN
#undef CAT
#undef CAT2
