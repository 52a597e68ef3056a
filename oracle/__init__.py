"""Plain CPU oracle of the SDM coalescence step.  Test infrastructure only:
imported by tests/, __graft_entry__.smoke() and bench.py's CPU legs, never by
the library."""
