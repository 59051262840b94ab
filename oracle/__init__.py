"""FP64 CPU oracle of the D2V16 multi-component DBM (arXiv 2006.15932).

Test infrastructure only: imported by the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``, never by the CUDA product path.
"""
