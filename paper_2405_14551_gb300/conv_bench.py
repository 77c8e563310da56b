"""Time one call of a surrogate convolution kernel on random BF16 data.

    python -m paper_2405_14551_gb300.conv_bench MODE NX NY NZ CIN COUT [REPS]

MODE: fwd (lbnn_conv3d_fwd), upcat (lbnn_conv3d_fwd_upcat with a third of
CIN at full resolution and the rest at half resolution) or wgrad
(lbnn_conv3d_wgrad).  3x3x3 taps, x and z periodic, y zero-padded.  Prints
the CUDA-event time of the last of REPS launches (default 3) and the FLOP
rate of the implicit GEMM (2 x 27 x CIN x COUT per voxel)."""
import ctypes
import sys


def main(argv):
    import torch
    from . import lbcg as L
    mode = argv[0]
    nx, ny, nz, cin, cout = (int(v) for v in argv[1:6])
    reps = int(argv[6]) if len(argv) > 6 else 3
    lib = L.load_library()
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream()
    sp = ctypes.c_void_p(st.cuda_stream)
    status = torch.zeros(4, dtype=torch.int32, device=dev)
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    nv = nx * ny * nz
    g = torch.Generator(device=dev).manual_seed(0)
    with torch.cuda.stream(st):
        w = (torch.randn(cout, 27, cin, device=dev, generator=g) * 0.05).to(torch.bfloat16)
        b = torch.zeros(cout, device=dev)
        cs = cin // 3 if mode == "upcat" else cin
        x = torch.randn(nv, cs, device=dev, generator=g).to(torch.bfloat16)
        x2 = torch.randn(nv // 8, cin - cs, device=dev, generator=g).to(torch.bfloat16) if mode == "upcat" else None
        y = torch.empty(nv, cout, device=dev, dtype=torch.bfloat16)
        gy = torch.randn(nv, cout, device=dev, generator=g).to(torch.bfloat16) if mode == "wgrad" else None
        dw = torch.zeros(cout, 27, cin, device=dev) if mode == "wgrad" else None
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for i in range(reps):
            if i == reps - 1:
                e0.record(st)
            if mode == "fwd":
                rc = lib.lbnn_conv3d_fwd(P(x), cin, P(w), 27, P(b), P(y), None, cout, 0, nx, ny, nz, 1, 5, 1,
                                         P(status), sp)
            elif mode == "upcat":
                rc = lib.lbnn_conv3d_fwd_upcat(P(x), cs, P(x2), cin - cs, P(w), P(b), P(y), None, cout, 0, nx, ny, nz,
                                               1, 5, 1, P(status), sp)
            elif mode == "wgrad":
                rc = lib.lbnn_conv3d_wgrad(P(gy), cout, P(x), cin, 27, P(dw), nx, ny, nz, 1, 5, 64, P(status), sp)
            else:
                raise SystemExit(f"unknown mode {mode}")
            if rc:
                raise SystemExit(f"{mode}: {lib.lb_last_error().decode()}")
        e1.record(st)
        st.synchronize()
    ms = e0.elapsed_time(e1)
    if int(status.sum().item()):
        raise SystemExit(f"{mode}: a kernel gave up a bounded wait (status {status.tolist()})")
    flop = 2.0 * nv * 27 * cin * cout
    print(f"{mode} {nx}x{ny}x{nz} {cin}->{cout}: {ms * 1e3:.1f} us, {flop / ms / 1e9:.1f} TFLOP/s")


if __name__ == "__main__":
    main(sys.argv[1:])
