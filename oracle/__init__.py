"""CPU oracle for TIM / TIM+ -- test infrastructure only.

Only the tests, the smoke check and the benchmark's CPU-baseline leg import this
package. It shares no code with the GPU library and never imports it.
"""
