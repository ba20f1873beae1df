"""Oracle package: plain, slow, single-threaded FP64 CPU reference of the tracking
hot path (element models, aperture loss, per-turn moments, wake, DA survival, MLP).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or run
anything in this package.  The product library (``paper_1710_07350_gb300``) never
imports it, and this package never imports the product library.
"""
