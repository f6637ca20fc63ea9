"""Run a named workload for profiling: build the model, warm up, run sweeps.

    python paper_1612_00595_gb300/profile_case.py --workload scale --warmup 3 --sweeps 2

Workloads: ``scale`` (4000 x 4000 km, 24 h, 1600 stations, float32),
``corner`` (1000 x 1000 km corner of the same density and record length,
100 stations: 0.7 GB of signals + variance, larger than L2), ``replay``
(1000 x 1000 km, 1 h, 100 stations, float64), ``train`` (the learned birth
network: ``--warmup`` then ``--sweeps`` training steps of 256 windows
simulated from the 1000 km, 1 h, 100-station float32 world).  ``--p-pair``
turns on joint moves of a pair of events, ``--sig-a`` / ``--p-arr`` latent
arrival times (the replay world generated with such offsets) and the
arrival-time move (float64 workloads).
"""
import argparse
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import worldgen  # noqa: E402


def world_for(name: str, sig_a: float = 0.0):
    if name == "scale":
        return worldgen.config_scale(seed=1000)
    if name == "corner":
        return worldgen.config_scale(seed=1000, side_regions=10)
    if name == "replay":
        return worldgen.config_replay(seed=1000, sig_a=sig_a)
    raise SystemExit("unknown workload " + name)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="corner")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--k", type=int, default=32)
    ap.add_argument("--p-pair", type=float, default=0.0)
    ap.add_argument("--sig-a", type=float, default=0.0)
    ap.add_argument("--p-arr", type=float, default=0.0)
    args = ap.parse_args()
    import paper_1612_00595_gb300 as cm
    if args.workload == "train":
        w = worldgen.config_learned(seed=1000)
        m = cm.create_model(None, w.stations, w.signals, cm.make_params(w.params, k_per_phase=args.k, seed=7,
                                                                        dtype=cm.F32))
        net = cm.Net(max_batch=256, seed=7)
        net.train(m, args.warmup, 256, 3e-4)
        loss = net.train(m, args.sweeps, 256, 3e-4)
        print("training steps %d  loss %.4f" % (args.warmup + args.sweeps, loss))
        net.destroy()
        m.destroy()
        return
    w = world_for(args.workload, args.sig_a)
    dtype = cm.F32 if w.signals.dtype == np.float32 else cm.F64
    m = cm.create_model(w.events, w.stations, w.signals, cm.make_params(w.params, k_per_phase=args.k, seed=7,
                                                                        dtype=dtype, p_pair=args.p_pair,
                                                                        sig_a=args.sig_a, p_arr=args.p_arr))
    if args.sig_a:
        m.set_arrival_offsets(w.offsets)
    m.partition_and_color(w.params.L, shift_mode=1)
    m.run_sweeps(args.warmup)
    m.sync()
    m.run_sweeps(args.sweeps)
    ev, ids, lp, st = m.read_state()
    print("events %d  proposals %d  accepted %s  pair %s  launches %d" % (
        len(ev), sum(st["proposed"]) + st["pair"][0] + st["arrival"][0], st["accepted"], st["pair"],
        st["kernel_launches"]))
    m.destroy()


if __name__ == "__main__":
    main()
