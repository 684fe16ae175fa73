"""Run by test_gpu_check_build.py in a process of its own with
AIM_LIBRARY=libaim_check.so: products in every precision (one and many
right-hand sides), the product without allocation, a packed product and a
solve through the index-checking debug build, each against the oracle or the
same build's reference path at the parity tolerances.  Any failed index check
makes the call return AIM_EINVAL, which raises here.  Prints "ok" at the end."""

import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from aim_inputs import icosphere_frequency, icosphere_mesh, plate_mesh, random_complex, random_incidence  # noqa: E402
from oracle import aim as oaim  # noqa: E402
from oracle.rwg import RWG  # noqa: E402

import paper_1010_1456_gb300 as g  # noqa: E402

K0, H = 2 * np.pi, 0.1


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


def main():
    assert g._lib.LIB_PATH.endswith("libaim_check.so"), g._lib.LIB_PATH
    torch.cuda.set_device(0)
    cases = [(plate_mesh(1.0, 9), 1.0, 17), (icosphere_mesh(0.3, icosphere_frequency(0.3)), 0.6, 2)]
    ctxs = []
    for (v, t), alpha, mr in cases:
        ctx = g.aim_setup(v, t, K0, H, max_rhs=mr, precision=g.AIM_C64, cfie_alpha=alpha)
        op = oaim.AIMOperator(RWG(v, t), K0, H, 2, near_radius=3 * H, alpha=alpha)
        for nr in sorted({1, mr}):
            x = random_complex((nr, ctx.N), seed=nr)
            ref = op.matvec(x)
            xd = torch.from_numpy(x).cuda()
            y64 = g.aim_matvec(ctx, xd.to(torch.complex64), precision=g.AIM_C64).cpu().numpy()
            assert rel(y64, ref) <= 1e-5, ("c64", nr, rel(y64, ref))
            for prec in (g.AIM_C128, g.AIM_C128_F64):
                y = g.aim_matvec(ctx, xd, precision=prec).cpu().numpy()
                assert rel(y, ref) <= 1e-12, (prec, nr, rel(y, ref))
        x1 = torch.from_numpy(random_complex((1, ctx.N), seed=7)).to(torch.complex64).cuda()
        a = g.aim_matvec(ctx, x1, precision=g.AIM_C64)
        b = torch.empty_like(a)
        g.check(g.load().aim_matvec_c64_noalloc(ctx.handle, g._dev(x1, torch.complex64), g._dev(b, torch.complex64),
                                                1), "aim_matvec_c64_noalloc")
        torch.cuda.synchronize()
        assert rel(b.cpu().numpy(), a.cpu().numpy()) <= 1e-5
        ctxs.append(ctx)
    # a pack of two spheres (the CFIE one above and an EFIE one) and a solve through it
    v, t = icosphere_mesh(0.4, icosphere_frequency(0.4))
    other = g.aim_setup(v, t, K0, H, max_rhs=1, precision=g.AIM_C64)
    pack = g.aim_pack_create([ctxs[1], other], [2, 1])
    xs = [random_complex((2, ctxs[1].N), seed=3), random_complex((1, other.N), seed=4)]
    yp = g.aim_pack_matvec(pack, pack.pack([torch.from_numpy(x).cuda() for x in xs]).to(torch.complex64).contiguous(),
                           precision=g.AIM_C64)
    for i, (ctx, x) in enumerate(zip([ctxs[1], other], xs)):
        alone = g.aim_matvec(ctx, torch.from_numpy(x).cuda(), precision=g.AIM_C128).cpu().numpy()
        assert rel(pack.unpack(yp)[i].cpu().numpy(), alone) <= 1e-5, ("pack", i)
    kh, po = random_incidence(1, rng=np.random.default_rng(2))
    Vs = [g.aim_rhs_planewave(ctxs[1], kh, po), g.aim_rhs_planewave(other, kh[:1], po[:1])]
    X, info = g.aim_pack_solve(pack, pack.pack(Vs), tol=1e-6)
    assert info["converged"].all() and info["rel_res"].max() <= 1e-6
    pack.close()
    X, info = g.aim_solve(ctxs[0], g.aim_rhs_planewave(ctxs[0], kh, po), tol=1e-6)
    assert info["converged"].all()
    for c in ctxs + [other]:
        c.close()
    print("ok")


if __name__ == "__main__":
    main()
